// Shared definitions of the CUDA sources (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "fhtdp.h"

namespace fhtdp {

// Sentinel of a dead DP state: no admissible polyline continues from it.
// It never takes part in an addition.
template <typename T>
struct Dead;
template <>
struct Dead<int32_t> {
    __host__ __device__ static constexpr int32_t value() { return INT32_MIN; }
};
template <>
struct Dead<float> {
    __device__ static float value() { return __int_as_float(0xff800000u); }
};

// Shape of one image's problem.
struct Shape {
    int h, w, k, n, W, D;  // D = 2n - 1 displacement values
    int log2n;
    // Vertex domain [0, vw) of the standalone DP and read-back: w, or W when
    // vertices may lie in the zero padding right of the image (Sec. 2.2).
    int vw;
};

// The continuation window of every displacement: entry d + n - 1 holds the
// range [lo, hi] of next displacements e admissible after d.  The bend-angle
// windows of Sec. 2.3 (Fig. 5, Eqs. 6-7: |atan(e/n) - atan(d/n)| <= gamma)
// and the integer bend limit |e - d| <= B are both such tables.  Passed to
// kernels by value.
constexpr int kMaxD = 511;
struct WindowTable {
    int16_t lo[kMaxD], hi[kMaxD];
    int n;
    int maxlen;  // the longest window, hi - lo + 1
};
// Fills *t for bands of n rows; false if gamma is negative or not finite.
bool make_angle_table(int n, double gamma, WindowTable *t);
// The integer bend limit as a table (B >= 0).
void make_bend_table(int n, int B, WindowTable *t);

// Largest half-width of the row smoothing (binomial weights up to C(24, 12)).
constexpr int kMaxGaussR = 12;

// Host helpers (api.cu).
int set_error(int code, const char *fmt, ...);
// Clears the calling thread's last error message (every entry point starts so).
void clear_error();
// Checks a launch and counts it (fhtdp_launch_count).
int launched(const char *what);
int cuda_status(cudaError_t err, const char *what);
bool make_shape(int h, int w, int k, Shape *out);

// Kernels launched by the API layer.
template <typename In, typename Acc>
int launch_fht_stages(const In *img, int pitch, const Shape &s, Acc *hough, Acc *tmp,
                      cudaStream_t stream);
// A point P = (xp, j*n) on the upper border of band j (j = k: the bottom
// border) that the polyline must pass (Subproblems 2-3): the DP marks every
// state whose vertex on that border is not xp dead.
struct PointMask {
    int j, xp;
};
template <typename Acc>
int launch_dp_inplace(Acc *hv, const Shape &s, int B, cudaStream_t stream,
                      const PointMask *pm = nullptr);
// The read-back with a grid-wide argmax into *key (zero before the call).
template <typename Acc>
int launch_backtrack_key(const Acc *V, const Shape &s, int B, unsigned long long *key,
                         int32_t *x_out, int32_t *d_out, Acc *score_out, cudaStream_t stream);
template <typename Acc>
int launch_backtrack(const Acc *V, const Shape &s, int B, int32_t *x_out, int32_t *d_out,
                     Acc *score_out, cudaStream_t stream);

// The main problem (Sec. 2.3): row smoothing into a dense [h][w] image
// (int32 for integer images, float for float ones), the DP with bend-angle
// windows, and its read-backs.
template <typename In, typename Acc>
int launch_gauss_rows(const In *img, int pitch, int h, int w, int r, Acc *out,
                      cudaStream_t stream);
// The band FHTs of the smoothed image without storing it: the smoothing is
// fused into the first level (bands of n >= 2 rows).
template <typename In, typename Acc>
int launch_fht_stages_gauss(const In *img, int pitch, const Shape &s, int r, Acc *hough, Acc *tmp,
                            cudaStream_t stream);
// The DP over any window table (int32 or float values), in place, with an
// optional through-point restriction.
template <typename Acc>
int launch_dp_window(Acc *hv, const Shape &s, const WindowTable &t, cudaStream_t stream,
                     const PointMask *pm = nullptr);
template <typename Acc>
int launch_backtrack_angle_key(const Acc *V, const Shape &s, const WindowTable &t,
                               unsigned long long *key, int32_t *x_out, int32_t *d_out,
                               Acc *score_out, cudaStream_t stream);
template <typename Acc>
int launch_backtrack_angle(const Acc *V, const Shape &s, const WindowTable &t, int32_t *x_out,
                           int32_t *d_out, Acc *score_out, cudaStream_t stream);
size_t angle_workspace_bytes(const Shape &s);
size_t through_workspace_bytes(const Shape &s);
// The method with vertices anywhere in [0, W) (s.vw = W): the standalone
// FHT, DP and key read-back.
int detect_padded(const void *img, int dtype, int pitch, const Shape &s, int B, int32_t *x_out,
                  int32_t *d_out, void *score_out, void *ws, cudaStream_t stream);
// Two different extreme polylines: the optimum and the best one whose top
// vertex is at least sep columns from the optimum's (outputs [2][...]).
int detect_two(const void *img, int dtype, int pitch, const Shape &s, int B, int sep,
               int32_t *x_out, int32_t *d_out, void *score_out, void *ws, cudaStream_t stream);
// The argmax of V_0 over the columns at least sep from the top vertex that
// key1 encodes (nothing when key1 is 0), into *key2 (zero before the call).
template <typename Acc>
int launch_argmax_apart(const Acc *V, const Shape &s, const unsigned long long *key1, int sep,
                        unsigned long long *key2, cudaStream_t stream);
// The read-back from an argmax key with the integer bend limit.
template <typename Acc>
int launch_readback_key(const Acc *V, const Shape &s, int B, const unsigned long long *key,
                        int32_t *x_out, int32_t *d_out, Acc *score_out, cudaStream_t stream);
// dst[x][y] = src[y][x] (Sec. 3, Fig. 7: mostly horizontal curves).
template <typename T>
int launch_transpose(const T *src, int h, int w, int pitch, T *dst, int dpitch,
                     cudaStream_t stream);
int detect_through(const void *img, int dtype, int pitch, const Shape &s, int B,
                   const PointMask &pm, int32_t *x_out, int32_t *d_out, void *score_out,
                   void *ws, cudaStream_t stream);
int detect_angle(const void *img, int dtype, int pitch, const Shape &s, int r,
                 const WindowTable &t, int32_t *x_out, int32_t *d_out, void *score_out,
                 void *ws, cudaStream_t stream, const PointMask *pm = nullptr);

}  // namespace fhtdp
