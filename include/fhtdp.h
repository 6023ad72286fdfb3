/*
 * fhtdp: detection of end-to-end curves of limited curvature on one GB300.
 *
 * C ABI of the library (libfhtdp.so).  It implements the data-parallel core
 * of "A Method of Detecting End-To-End Curves of Limited Curvature"
 * (Panfilova, Aliev, Kunina, Postnikov, Nikolaev, arXiv 1912.01884): a Fast
 * Hough Transform of each of the k horizontal bands of an image (Sec. 2.1), a
 * bottom-up max-plus dynamic programme over the bands with a bend limit
 * (Sec. 2.2-2.3, Eqs. 3-4), and the read-back of the best k-link polyline
 * (Eq. 5 and the main problem's steps 2-3); and around it the paper's main
 * problem with row smoothing and a bend angle (Sec. 2.3), the polyline
 * through a given point (Subproblems 2-3), vertices in the zero padding,
 * mostly horizontal curves and two different polylines (Sec. 3).
 *
 * Conventions shared by every call
 *   h, w      image height and width in pixels; h = k * n with n a power of
 *             two (n rows per band, 1 <= n <= 256); 1 <= w.
 *   pitch     row stride of the image in ELEMENTS (>= w).
 *   dtype     FHTDP_U8 (uint8 pixels), FHTDP_I32 (int32 pixels) or FHTDP_F32
 *             (float pixels).  Integer images accumulate in int32 (exact as
 *             long as max|pixel| * h < 2^31, which the caller guarantees);
 *             float images accumulate in float32 with a fixed summation tree
 *             (each Hough value is the pairwise sum, top half + bottom half,
 *             of its band rows).
 *   W = w + n the width of a band after it is zero-padded on the right by
 *             h/k columns (Sec. 2.1).
 *   A link of band i joins column x_i on the band's first row to column
 *   x_{i+1} = x_i + d_i on its last row, |d_i| <= n-1 (the paper's shift of
 *   Eq. 1 is n - d_i); the pixels it covers follow the FHT's dyadic pattern.
 *   Every vertex x_0..x_k lies in [0, w) (fhtdp_detect_polyline_padded:
 *   [0, w + n)).  The bend limit is the integer range |d_{i+1} - d_i| <= B
 *   (B >= 2n-2 means unrestricted, Sec. 2.2); the main-problem calls
 *   (*_angle) limit the bend angle instead (Sec. 2.3, Eqs. 6-7).
 *   Among optimal polylines the lexicographically smallest
 *   (x_0, d_0, ..., d_{k-1}) is returned (d ordered numerically).
 *   Scores are int32 for integer images and float for float images.
 *
 * Memory and streams
 *   Every pointer argument named img, hough, V, ws, x_out, d_out, score_out
 *   is DEVICE memory owned by the caller; the library never allocates device
 *   memory and never synchronises the stream.  All work is enqueued on
 *   `stream` (0 = legacy default stream) and results are valid once the
 *   stream has reached them.
 *
 * Errors
 *   Every call returns an fhtdp status.  Bad arguments return FHTDP_EINVAL
 *   before anything is enqueued; a workspace that is too small returns
 *   FHTDP_EWORKSPACE; a CUDA launch error returns FHTDP_ECUDA.  The message of
 *   the last failure on the calling thread is returned by fhtdp_last_error().
 *   No C++ exception crosses this interface.
 */
#ifndef FHTDP_H
#define FHTDP_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

enum fhtdp_status {
    FHTDP_OK = 0,
    FHTDP_EINVAL = 1,     /* invalid argument (nothing was enqueued) */
    FHTDP_EWORKSPACE = 2, /* workspace missing or smaller than required */
    FHTDP_ECUDA = 3,      /* a CUDA call failed; see fhtdp_last_error() */
    FHTDP_ETIMEOUT = 4    /* a bounded device-side wait gave up */
};

enum fhtdp_dtype { FHTDP_U8 = 0, FHTDP_I32 = 1, FHTDP_F32 = 2 };

/* Message of the last failed call on this thread ("" if none).  The string
 * stays valid until the next call on the same thread. */
const char *fhtdp_last_error(void);

/* Library ABI version (major * 100 + minor). */
int fhtdp_version(void);

/* Number of CUDA kernel launches the library has enqueued in this process
 * (all threads, all devices), for accounting by benchmarks. */
uint64_t fhtdp_launch_count(void);

/* Bytes of a Hough / DP-value array of the given shape:
 * k * 2 * n * (w + n) elements of 4 bytes (int32 or float).
 * Returns 0 for invalid shapes. */
size_t fhtdp_hough_bytes(int dtype, int h, int w, int k);

/* Sec. 2.1 (Subproblem 1): the Hough images H_0..H_{k-1} of the k
 * zero-padded bands, for mostly vertical lines of both slope signs.
 *   img    [h rows][pitch] pixels of `dtype` (device).
 *   hough  output, [k][2][n][W] int32 (integer images) or float (float
 *          images), x fastest (device, fhtdp_hough_bytes()).  Element
 *          [i][0][s][x] is the sum along the line from (x, first row of band
 *          i) moving s columns right over the band; [i][1][s][x] the same
 *          moving left; columns are taken modulo W (cyclic FHT), so for
 *          x in [0, w) and an end column inside the image it is the plain sum.
 *   ws     device workspace of at least fhtdp_fht_workspace_bytes() bytes
 *          (stage ping-pong buffer), overwritten.
 */
size_t fhtdp_fht_workspace_bytes(int dtype, int h, int w, int k);
int fhtdp_fht_bands(const void *img, int dtype, int h, int w, int pitch, int k,
                    void *hough, void *ws, size_t ws_bytes, cudaStream_t stream);

/* Sec. 2.2-2.3, Eqs. 3-4: the bottom-up DP, in place over the Hough images
 * exactly as the paper updates H_{i-1} with the best continuation.
 *   hough  in: output of fhtdp_fht_bands.  out: DP values V_i(x, d) = best
 *          sum of a polyline that starts with link (x, d) in band i and ends
 *          on the image's last row; V_i(x, +s) at [i][0][s][x], V_i(x, -s)
 *          at [i][1][s][x] (s = 0 stored in both), x in [0, w).  Dead states
 *          (end vertex outside [0, w), or no admissible continuation) and
 *          the padding columns [w, W) hold INT32_MIN / -infinity.
 *   B      bend limit, >= 0.
 */
int fhtdp_polyline_dp(void *hough, int dtype, int h, int w, int k, int B, cudaStream_t stream);

/* Eq. 5 and the main problem, steps 2-3: the best top point and the read-back
 * of its polyline from DP values laid out as fhtdp_polyline_dp leaves them.
 *   x_out  k+1 int32 vertices x_0..x_k (device).
 *   d_out  k int32 displacements d_i = x_{i+1} - x_i (device).
 *   score_out  one int32 (integer images) or float (float images) (device).
 */
int fhtdp_backtrack(const void *V, int dtype, int h, int w, int k, int B,
                    int32_t *x_out, int32_t *d_out, void *score_out, cudaStream_t stream);

/* The whole method on one image (Sec. 2.1-2.3 and the main problem): the
 * band FHTs, the bend-limited DP and the read-back, through the fused engine
 * (the Hough images never reach global memory).
 *   ws     device workspace of at least fhtdp_workspace_bytes() bytes.
 *   Outputs as for fhtdp_backtrack.  Returns FHTDP_ETIMEOUT if a device-side
 *   dependency wait gave up (the outputs are then undefined).
 */
size_t fhtdp_workspace_bytes(int dtype, int h, int w, int k, int B);
int fhtdp_detect_polyline(const void *img, int dtype, int h, int w, int pitch, int k, int B,
                          int32_t *x_out, int32_t *d_out, void *score_out,
                          void *ws, size_t ws_bytes, cudaStream_t stream);

/* fhtdp_detect_polyline without a caller workspace.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory (hosts that own all device memory themselves, or real-time loops in
 * which a cudaMalloc, which may synchronise the device, is not allowed).  It
 * allocates nothing: its scratch is a fixed array of
 * FHTDP_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads
 * the library holds until the process exits.  Arguments, outputs and results
 * are those of fhtdp_detect_polyline.
 *   - Images whose scratch (fhtdp_workspace_bytes) exceeds the array are
 *     rejected with FHTDP_EWORKSPACE before anything is enqueued (a 2048x2048
 *     uint8 image with 128-row bands needs about 12.5 MiB).
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *   - All calls share the one array, and it keeps the last call's contents;
 *     each call clears the parts that must start at zero.  Calls whose work
 *     overlaps on the GPU (different streams, or different host threads on the
 *     same device without ordering) race on the array: order them on one
 *     stream.
 *   - A bounded device-side wait that gave up is reported by
 *     fhtdp_detect_polyline_noalloc_status, not by fhtdp_workspace_status. */
#define FHTDP_NOALLOC_SCRATCH_BYTES (16u << 20)
int fhtdp_detect_polyline_noalloc(const void *img, int dtype, int h, int w, int pitch, int k,
                                  int B, int32_t *x_out, int32_t *d_out, void *score_out,
                                  cudaStream_t stream);

/* The status of the last fhtdp_detect_polyline_noalloc run on the current
 * device, read from the control block of the built-in scratch: FHTDP_OK, or
 * FHTDP_ETIMEOUT if one of its bounded device-side waits gave up (its outputs
 * are then undefined).  Synchronises `stream`, on which that run was
 * enqueued.  The paper has no counterpart; this exists for the same callers
 * as fhtdp_detect_polyline_noalloc, which have no workspace of their own to
 * pass to fhtdp_workspace_status. */
int fhtdp_detect_polyline_noalloc_status(cudaStream_t stream);

/* ------------------------------------------------------------------------
 * The main problem of Sec. 2.3 (the Welsh M-estimate of a k-link polyline
 * with a bending-angle limit).  Step 1 convolves every row with a discrete
 * Gaussian; steps 2-3 run the DP and the read-back with the bend-angle
 * windows of Eqs. 6-7 instead of the integer limit B.
 *
 *   Gaussian  the binomial weights C(2r, r+t), |t| <= r (the discrete
 *             Gaussian of variance r/2), not normalised: every polyline sum
 *             is scaled by the same 4^r, which leaves the optimum unchanged
 *             and keeps integer arithmetic exact.  Pixels outside the row
 *             count as zero.  0 <= r <= 12; r = 0 is no smoothing.
 *   gamma     the largest bending angle in radians (>= 0, finite).  A link
 *             of displacement d has inclination atan(d/n) from the vertical;
 *             the next link's e is admissible when
 *             |atan(e/n) - atan(d/n)| <= gamma, evaluated in double (Fig. 5,
 *             Eqs. 6-7; the pi/4 limit of Eqs. 6-7 is |e| <= n-1).
 *             gamma = 0 keeps the displacement fixed; gamma >= pi/2 admits
 *             every e.
 *   dtype     FHTDP_U8 or FHTDP_I32: sums are int32; uint8 images need
 *             255 * 4^r * h < 2^31 (checked); int32 images need
 *             max|pixel| * 4^r * h < 2^31 (the caller guarantees it).
 *             FHTDP_F32: everything in float32, each smoothing product
 *             weight * pixel rounded and added in the order t = -r..r, the
 *             FHT sums in the tree of fhtdp_fht_bands, the argmax decisions
 *             taken on the float32 values.
 *   Scores are int32 (integer images) or float (float images) and refer to
 *   the smoothed image.  Ties are broken as in fhtdp_detect_polyline (the
 *   lexicographically smallest polyline).
 * ---------------------------------------------------------------------- */
/* The window of every displacement, on the host: lohi[2n-1][2] (HOST
 * memory, written by the call), row d + n - 1 = {lo(d), hi(d)}.  n is a
 * power of two in [1, 256]. */
int fhtdp_angle_window(int n, double gamma, int32_t *lohi);

/* Step 1: out[y][x] = sum_t C(2r, r+t) img[y][x+t] (device; out is a dense
 * [h][w] array, pitch w, of int32 for integer images or float for float
 * images, that must not overlap img). */
int fhtdp_gauss_rows(const void *img, int dtype, int h, int w, int pitch, int r, void *out,
                     cudaStream_t stream);

/* Step 2: the DP of fhtdp_polyline_dp over Hough images (int32, or float for
 * FHTDP_F32; laid out as fhtdp_fht_bands leaves them), in place, with the
 * bend-angle windows. */
int fhtdp_polyline_dp_angle(void *hough, int dtype, int h, int w, int k, double gamma,
                            cudaStream_t stream);

/* Step 3: the read-back of fhtdp_backtrack with the bend-angle windows. */
int fhtdp_backtrack_angle(const void *V, int dtype, int h, int w, int k, double gamma,
                          int32_t *x_out, int32_t *d_out, void *score_out, cudaStream_t stream);

/* Steps 1-3 on one image: smoothing, band FHTs, the angle DP and the
 * read-back.  ws: device workspace of at least fhtdp_angle_workspace_bytes()
 * bytes (0 for invalid arguments).  Outputs as for fhtdp_backtrack. */
size_t fhtdp_angle_workspace_bytes(int dtype, int h, int w, int k, int r);
int fhtdp_detect_polyline_angle(const void *img, int dtype, int h, int w, int pitch, int k,
                                int r, double gamma, int32_t *x_out, int32_t *d_out,
                                void *score_out, void *ws, size_t ws_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Subproblems 2-3 (Sec. 2.2-2.3): the extreme polyline through a given point
 * P = (xp, j*n) on the upper border of band j, 0 <= j <= k (j = k is the
 * image's bottom border), 0 <= xp < w.  The result is the best admissible
 * polyline (bend limit B at every vertex, P included) with x_j = xp, the
 * lexicographically smallest among the optimal ones; B >= 2n-2 is
 * Subproblem 2 (no bend limit).  The paper finds the part above P by
 * flipping the top bands about Ox; one DP over all bands with the states of
 * P's band off xp marked dead reaches the same optimum.
 *   dtype  any of the three; float32 images are computed and decided in
 *          float32 as in fhtdp_detect_polyline.
 *   ws     device workspace of at least fhtdp_through_workspace_bytes()
 *          bytes (0 for invalid arguments).  Outputs as for fhtdp_backtrack.
 * ---------------------------------------------------------------------- */
size_t fhtdp_through_workspace_bytes(int dtype, int h, int w, int k);

/* Subproblem 3 with the bend angle (Sec. 2.3): the best polyline through P =
 * (xp, j*n) whose consecutive links bend by at most gamma, on the image with
 * its rows smoothed (half-width r; r = 0 is none).  r, gamma, dtype and the
 * score as for fhtdp_detect_polyline_angle, j and xp as for
 * fhtdp_detect_through_point; ws of at least fhtdp_angle_workspace_bytes(). */
int fhtdp_detect_through_point_angle(const void *img, int dtype, int h, int w, int pitch, int k,
                                     int r, double gamma, int j, int xp, int32_t *x_out,
                                     int32_t *d_out, void *score_out, void *ws, size_t ws_bytes,
                                     cudaStream_t stream);
int fhtdp_detect_through_point(const void *img, int dtype, int h, int w, int pitch, int k, int B,
                               int j, int xp, int32_t *x_out, int32_t *d_out, void *score_out,
                               void *ws, size_t ws_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Vertices in the zero padding (Sec. 2.2: the Hough columns run over
 * [0, w + h/k - 1]; Sec. 2.1 extends every band by n zero columns on the
 * right).  As fhtdp_detect_polyline, but every vertex may lie anywhere in
 * [0, W), W = w + n: the pixels a link covers right of the image count as
 * zero, so a curve that runs off the right edge can be followed.  Runs the
 * standalone kernels.  dtype any of the three; ws of at least
 * fhtdp_through_workspace_bytes() bytes.  Outputs as for fhtdp_backtrack.
 * ---------------------------------------------------------------------- */
int fhtdp_detect_polyline_padded(const void *img, int dtype, int h, int w, int pitch, int k,
                                 int B, int32_t *x_out, int32_t *d_out, void *score_out,
                                 void *ws, size_t ws_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Two different extreme polylines (Sec. 3, Figs. 6d and 7a, where the paper
 * shows two and states no rule).  The first is the optimum of
 * fhtdp_detect_polyline; the second is the best admissible polyline whose top
 * vertex x_0 lies at least sep (>= 1) columns from the first's (suppression
 * on x_0), the lexicographically smallest among its optima.  When no column
 * is far enough, the second has x = -1 everywhere and score INT32_MIN (or
 * -infinity for float images).
 *   dtype  any of the three.
 *   x_out [2][k+1], d_out [2][k], score_out [2] int32 or float (device).
 *   ws     device workspace of at least fhtdp_two_workspace_bytes() bytes.
 * ---------------------------------------------------------------------- */
size_t fhtdp_two_workspace_bytes(int dtype, int h, int w, int k);
int fhtdp_detect_two_polylines(const void *img, int dtype, int h, int w, int pitch, int k, int B,
                               int sep, int32_t *x_out, int32_t *d_out, void *score_out,
                               void *ws, size_t ws_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Mostly horizontal curves (Sec. 3, Fig. 7): the method on the transposed
 * image.  The bands are the image's k vertical strips of n = w/k columns (n a
 * power of two, 1 <= n <= 256); link i joins row y_i on the strip's first
 * column to row y_{i+1} = y_i + d_i on its last column, |d_i| <= n-1, every
 * y_i in [0, h).  The image is transposed into the workspace and run through
 * the fused engine, so results, ties and errors are those of
 * fhtdp_detect_polyline on the transposed image (dtype any of the three).
 *   y_out [k+1], d_out [k], score_out [1] (device).
 *   ws     device workspace of at least fhtdp_horizontal_workspace_bytes();
 *          fhtdp_workspace_status is not available for these calls.
 * ---------------------------------------------------------------------- */
size_t fhtdp_horizontal_workspace_bytes(int dtype, int h, int w, int k, int B);
/* dst[x][y] = src[y][x]: src [h][pitch], dst [w][dpitch] (dpitch >= h), both
 * device, not overlapping.  A batch of mostly horizontal images is
 * transposed with this call and then run as one fhtdp_batch_run. */
int fhtdp_transpose(const void *src, int dtype, int h, int w, int pitch, void *dst, int dpitch,
                    cudaStream_t stream);
int fhtdp_detect_polyline_horizontal(const void *img, int dtype, int h, int w, int pitch, int k,
                                     int B, int32_t *y_out, int32_t *d_out, void *score_out,
                                     void *ws, size_t ws_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Learned window proposal (no counterpart in the paper): a 4-layer,
 * 32-channel 3x3 CNN on the 4x4-downsampled image predicts, for each band, a
 * bin of 4 displacements; the DP then searches only a window around it
 * (fhtdp_image.d_window), with the full DP as the fallback.  Activations are
 * NHWC bf16 (C = 32; the input has C = 1), weights bf16 [tap = 3*ky+kx][ci][co]
 * (the single-channel first layer: [16][32], taps 9..15 zero), FP32
 * accumulation on the tensor cores, FP32 master weights.  All pointers are
 * device memory owned by the caller; w must be a multiple of 64 and the
 * dilation at most 8.
 * ---------------------------------------------------------------------- */
/* uint8 [n][h][w] -> bf16 [n][h/4][w/4], the 4x4 mean divided by 255. */
int fhtdp_cnn_downsample4(const uint8_t *img, int n, int h, int w, void *out, cudaStream_t stream);
/* y = act(conv3x3_dil(x, wt) + bias), act = ReLU when relu != 0; cin 1 or 32,
 * cout 32, zero padding ("same").  32 input channels run on tcgen05.mma
 * (persistent CTAs over tiles of 128 pixels x 32 channels, K = 9 x 32, FP32
 * accumulators in tensor memory); a bounded wait for the MMAs that gives up
 * records FHTDP_ETIMEOUT for fhtdp_cnn_status. */
int fhtdp_cnn_conv3x3(const void *x, int cin, int n, int h, int w, int dil, const void *wt,
                      const float *bias, int relu, void *y, cudaStream_t stream);
/* Device status of the tensor-core convolutions since the last clear: 0, or
 * FHTDP_ETIMEOUT when a wait for the MMAs gave up (the results are then
 * undefined); clear != 0 resets it.  Synchronises the device (not for use
 * under stream capture).  Returns a negative FHTDP_ECUDA-coded value only if
 * the status cannot be read. */
int fhtdp_cnn_status(int clear);
/* dx = gradient of a 32-channel layer's input from the gradient dz of its
 * pre-activation output; wflip is caller scratch of 9*32*32 bf16. */
int fhtdp_cnn_conv3x3_dgrad(const void *dz, int n, int h, int w, int dil, const void *wt,
                            void *wflip, void *dx, cudaStream_t stream);
/* dy *= (y > 0): the ReLU of a layer, in place, from its output y. */
int fhtdp_cnn_relu_backward(const void *y, void *dy, long long count, cudaStream_t stream);
/* dw += sum over pixels of x(shifted by the tap) * dz (FP32 [taps][cin][32]),
 * db += sum of dz (FP32 [32], may be NULL).  Accumulates: clear first.  32
 * input channels run on tcgen05.mma (the pixels as K, FP32 accumulators in
 * tensor memory; the sums' order across CTAs varies between runs). */
int fhtdp_cnn_conv3x3_wgrad(const void *x, int cin, int n, int h, int w, int dil, const void *dz,
                            float *dw, float *db, cudaStream_t stream);
/* Band head: pooled[n][b][c] = log-sum-exp of logits[n][rows of band b][:][c];
 * loss += scale * cross-entropy(softmax(pooled), labels[n][b]) (labels may
 * be NULL), dlogits = its gradient (may be NULL), pred[n][b] = argmax_c
 * pooled (may be NULL). */
int fhtdp_cnn_band_head(const void *logits, int n, int h, int w, int bands,
                        const int32_t *labels, float scale, void *dlogits, float *loss,
                        int32_t *pred, cudaStream_t stream);
/* One Adam step (step >= 1) on FP32 parameters p with moments m, v and
 * gradient g; also writes the bf16 copy wb (may be NULL). */
int fhtdp_cnn_adam(float *p, float *m, float *v, const float *g, int count, float lr, float b1,
                   float b2, float eps, int step, void *wb, cudaStream_t stream);
/* bf16 copy of FP32 values. */
int fhtdp_cnn_to_bf16(const float *src, void *dst, int count, cudaStream_t stream);
/* Pruned-DP windows from predicted bins: bin c covers displacements d with
 * d + 64 in [4c, 4c+3]; win[i] = that range widened by `margin` on each side,
 * clipped to [-(n-1), n-1]. */
int fhtdp_cnn_bin_windows(const int32_t *pred, int count, int n, int margin, int32_t *win,
                          cudaStream_t stream);

/* Status of the last detection run that used this workspace (a single image
 * or a batch): FHTDP_OK, or FHTDP_ETIMEOUT if one of its bounded device-side
 * waits gave up (its outputs are then undefined).  Synchronises `stream`
 * (one 4-byte device-to-host copy). */
int fhtdp_workspace_status(const void *ws, cudaStream_t stream);

/* Test hook for failure detection (no counterpart in the paper): the next
 * fused-engine run started from this host thread (fhtdp_detect_polyline or
 * fhtdp_batch_run) never publishes the window maxima of column tile `tile` of
 * band `band` of its first image, and its device-side waits give up after
 * `wait_cycles` SM cycles instead of about two seconds.  The run then ends with
 * FHTDP_ETIMEOUT in fhtdp_workspace_status and undefined outputs; the CUDA
 * context stays usable.  Nothing faults or hangs. */
void fhtdp_debug_inject(int band, int tile, long long wait_cycles);

/* ------------------------------------------------------------------------
 * Batches: many images of different h, w, k and B (one pixel type) in ONE
 * persistent kernel launch.  Work items (image, band, column tile) are taken
 * from a device-side queue, so the band chains of different images overlap
 * and the GPU stays busy; a run is one memset and one kernel launch and may
 * be captured in a CUDA graph.  Each image's result is the same as
 * fhtdp_detect_polyline's.
 * ---------------------------------------------------------------------- */
typedef struct fhtdp_image {
    const void *img;     /* device pixels [h][pitch] of the batch's dtype */
    int h, w, pitch, k, B;
    int32_t *x_out;      /* device, k+1 vertices */
    int32_t *d_out;      /* device, k displacements */
    void *score_out;     /* device, one int32 (integer images) or float */
    /* Optional (NULL = none): device [k][2] int32, the allowed displacements
     * [lo_i, hi_i] of each band's link.  With it the DP searches only those
     * links (the pruned DP of the learned proposal, which the paper does not
     * have) and returns the best polyline inside the windows; if there is none,
     * the score is INT32_MIN / -infinity and every vertex -1.  Bands of at most
     * 128 rows. */
    const int32_t *d_window;
} fhtdp_image;

typedef struct fhtdp_batch_plan fhtdp_batch_plan;

/* Validates every image (FHTDP_EINVAL names the first bad one), lays out its
 * scratch and orders the work queue.  The plan is a host object owned by the
 * caller (fhtdp_batch_plan_destroy); `images` is copied. */
int fhtdp_batch_plan_create(const fhtdp_image *images, int count, int dtype,
                            fhtdp_batch_plan **plan_out);
/* Device workspace the plan needs (bytes). */
size_t fhtdp_batch_workspace_bytes(const fhtdp_batch_plan *plan);
/* Binds the plan to a workspace: enqueues one host-to-device copy of the
 * image table into `ws` (from memory held by the plan; keep the plan alive
 * until the copy has run).  Call once per workspace, before the runs. */
int fhtdp_batch_upload(fhtdp_batch_plan *plan, void *ws, size_t ws_bytes, cudaStream_t stream);
/* Runs the whole batch on `stream`: one memset and one kernel launch. */
int fhtdp_batch_run(const fhtdp_batch_plan *plan, void *ws, cudaStream_t stream);
/* Number of work items (image, band, column tile) of a run. */
long long fhtdp_batch_items(const fhtdp_batch_plan *plan);
/* Tunes the plan on its bound workspace (after fhtdp_batch_upload) by timing
 * runs: the call runs the batch `reps` times (plus one warm-up) per candidate
 * and keeps the fastest of each choice in turn:
 *   1. the work-queue schedule: groups of images whose band levels hold about
 *      `target` column tiles and advance together, or band chains (an active
 *      set of about `target` tiles per step that images join, most bands
 *      first, as others finish), with the images of 256-row bands spread
 *      evenly through that join order or not, and advancing every step or
 *      every second step; widths from half to six times the SM count and the
 *      whole batch;
 *   2. for each band height of uint8 images, the column tile width of its
 *      work items (128, or 256 for bands of at most 64 rows) and the number
 *      of FHT levels done in registers before the shared-memory merges (2 or
 *      3; 256-row bands: of their 128-row halves);
 *   3. the schedule again.
 * It uploads the chosen layout and queue, and writes the width to
 * *target_out (may be NULL); fhtdp_batch_choice reports the rest.  The
 * outputs are those of an ordinary run.  It synchronises `stream` (not for use
 * under stream capture).  The paper has no counterpart: this tunes the GPU
 * schedule of its method, not the method. */
int fhtdp_batch_autotune(fhtdp_batch_plan *plan, void *ws, int reps, cudaStream_t stream,
                         long long *target_out);
/* The plan's current choices: the queue schedule (*mode: 0 groups, 1 band
 * chains, 2 band chains with the 256-row-band images spread, 3 band chains
 * with 256-row bands every second step, 4 both) and width, and for its images of band height n the column tile
 * width and register FHT depth (0 and 0 when it has none).  Any pointer may
 * be NULL.  The paper has no counterpart (see fhtdp_batch_autotune). */
int fhtdp_batch_choice(const fhtdp_batch_plan *plan, int n, int *mode, long long *target,
                       int *tile, int *depth);
/* Sets, by hand, the column tile width and register FHT depth of the plan's
 * uint8 images of band height n (the choices of step 2 of
 * fhtdp_batch_autotune; FHTDP_EINVAL for one that band height does not
 * allow) and enqueues the upload of the new layout and queue into the bound
 * workspace `ws`.  The paper has no counterpart (see fhtdp_batch_autotune). */
int fhtdp_batch_configure(fhtdp_batch_plan *plan, void *ws, int n, int tile, int depth,
                          cudaStream_t stream);
/* Sec. 2.3, Eqs. 6-7 (main problem step 2): the plan's runs take the
 * bend-angle windows of gamma (radians, >= 0) instead of the images' integer
 * bend limits: after a link of displacement d the next one's e satisfies
 * |atan(e/n) - atan(d/n)| <= gamma (the table of fhtdp_angle_window), and the
 * polyline read back is the same as fhtdp_polyline_dp_angle +
 * fhtdp_backtrack_angle give.  The images are the rows already smoothed
 * (fhtdp_gauss_rows, step 1): int32 or float32, all of one band height n in
 * 2..128.  Host only (no device work); FHTDP_EINVAL otherwise.  All the
 * images' band chains then run in one persistent launch: the window maxima
 * come from maxima of a fixed half-width that cover every window. */
int fhtdp_batch_angle(fhtdp_batch_plan *plan, double gamma);
/* Sec. 2.2-2.3, Subproblems 2-3: the plan's runs find, for image i, the best
 * polyline through the point (points[2i + 1], points[2i] n) on band border
 * points[2i] (1..k; k is the image's bottom border; a point on the top border
 * is for fhtdp_detect_through_point), as fhtdp_detect_through_point does;
 * points[2i] < 0 leaves image i unrestricted.  `points` is host memory read
 * during the call ([count][2] int32, the images in the order given to
 * fhtdp_batch_plan_create).  uint8 images with at least two bands of at most
 * 128 rows only (FHTDP_EINVAL otherwise, and for a point outside [0, w) x
 * [1, k]).  Enqueues the upload of the image table into the bound workspace
 * `ws` on `stream`. */
int fhtdp_batch_points(fhtdp_batch_plan *plan, void *ws, const int32_t *points,
                       cudaStream_t stream);
void fhtdp_batch_plan_destroy(fhtdp_batch_plan *plan);

/* ------------------------------------------------------------------------
 * The learned window proposal in front of the exact method (the paper has
 * no counterpart).  A 4-layer, 32-channel CNN (3x3 convolutions with
 * dilations 1, 2, 4, 8, ReLU after the first three, bf16 weights on the
 * tensor cores with FP32 accumulation) reads the 4x4 mean-pooled image and
 * predicts, for every band, one of 32 bins of 4 displacements
 * (d + 64 in [4c, 4c + 3]); the DP then searches only a window around it.
 *
 * Parameter block (device, fhtdp_cnn_param_bytes() bytes, caller-owned): per
 * layer, each part from a 256-byte boundary, the FP32 weights [rows][32]
 * (layer 1: 16 rows = taps, rows 9..15 zero; layers 2-4: 9 taps x 32 input
 * channels), the FP32 bias [32], the Adam moments of the weights and of the
 * bias (first, second), and the bf16 copy of the weights the forward pass
 * reads.
 * ---------------------------------------------------------------------- */
size_t fhtdp_cnn_param_bytes(void);
/* He-normal weights (standard deviation sqrt(2 / fan_in), from a seeded
 * counter-based generator), zero biases and moments, bf16 copies. */
int fhtdp_cnn_init(void *params, unsigned long long seed, cudaStream_t stream);
/* Workspace of fhtdp_cnn_forward / _backward / _step for n images of h x w
 * pixels: the pooled input, the four layers' outputs, two gradient buffers
 * and the FP32 gradients. */
size_t fhtdp_cnn_workspace_bytes(int n, int h, int w);
/* Forward pass of n uint8 images [n][h][w] (device, contiguous; h and w
 * multiples of 4, w/4 a multiple of 64, (h/4) divisible by `bands`):
 * pred[n][bands] = the predicted bin of every band (log-sum-exp pooling of
 * the band's logits, then argmax), conf[n][bands] = its softmax probability
 * (may be NULL).  Leaves the activations in ws for fhtdp_cnn_backward. */
int fhtdp_cnn_forward(const void *params, const uint8_t *imgs, int n, int h, int w, int bands,
                      void *ws, size_t ws_bytes, int32_t *pred, float *conf,
                      cudaStream_t stream);
/* Backward pass after fhtdp_cnn_forward on the same ws: the mean softmax
 * cross-entropy of the pooled band logits against labels[n][bands] (bins,
 * device) into *loss (device, may be NULL), and every layer's FP32 gradient
 * into ws. */
int fhtdp_cnn_backward(const void *params, const int32_t *labels, int n, int h, int w, int bands,
                       void *ws, size_t ws_bytes, float *loss, cudaStream_t stream);
/* One Adam step (beta 0.9, 0.999, eps 1e-8; step >= 1) on the FP32
 * parameters with the gradients left in ws; refreshes the bf16 copies. */
int fhtdp_cnn_step(void *params, const void *ws, int n, int h, int w, float lr, int step,
                   cudaStream_t stream);

/* Learned detection of a batch of uint8 images of one shape, stored one after
 * the other ([count][h][w], pitch w; bands of at most 128 rows), through a
 * plan bound to a workspace like the batch plans:
 *   1. the CNN proposes every band's bin; the window is the bin's 4
 *      displacements widened by window_half on both sides;
 *   2. a pruned DP (one persistent launch) finds the best polyline inside
 *      the windows;
 *   3. an image falls back to the full DP when the pruned DP found no
 *      polyline, when the polyline touches a window edge that is not an edge
 *      of the displacement range, when its score is below the confidence
 *      margin, margin * h (a mean intensity per image row), or when the
 *      network gave some band's bin a softmax probability below min_conf;
 *      used_fallback[i] (device, may be NULL) records it;
 *   4. one more persistent launch runs the full DP of the images that fall
 *      back only (the others' work items are skipped), into the images'
 *      outputs; the others get the pruned result.
 * Everything is enqueued on `stream`, with no host synchronisation: the call
 * may be captured in a CUDA graph.  Images that fall back get exactly
 * fhtdp_detect_polyline's results. */
typedef struct fhtdp_learned_plan fhtdp_learned_plan;
int fhtdp_learned_plan_create(const fhtdp_image *images, int count, int window_half,
                              fhtdp_learned_plan **plan_out);
size_t fhtdp_learned_workspace_bytes(const fhtdp_learned_plan *plan);
/* Binds the plan to `ws` (uploads its tables; synchronises `stream`). */
int fhtdp_learned_upload(fhtdp_learned_plan *plan, void *ws, size_t ws_bytes,
                         cudaStream_t stream);
int fhtdp_detect_learned(fhtdp_learned_plan *plan, const void *params, float margin,
                         float min_conf, int32_t *used_fallback, void *ws, cudaStream_t stream);
/* FHTDP_ETIMEOUT if a bounded device wait of the last detect_learned on this
 * workspace gave up; synchronises `stream`. */
int fhtdp_learned_status(const fhtdp_learned_plan *plan, const void *ws, cudaStream_t stream);
void fhtdp_learned_plan_destroy(fhtdp_learned_plan *plan);

#ifdef __cplusplus
}
#endif

#endif /* FHTDP_H */
