// In-place DP over the Hough images and the read-back (the standalone
// fhtdp_polyline_dp / fhtdp_backtrack calls).
//
// Sec. 2.2-2.3, Eqs. 3-4: going up from the last band, every Hough cell
// (x, d) of band i is increased by the best admissible continuation in band
// i+1, i.e. the maximum of V_{i+1}(x + d, e) over the bend window
// |e - d| <= B.  Eq. 5 and the main problem's steps 2-3: the best top point
// is the maximum of V_0, and the polyline is read back band by band.
//
// These kernels keep the paper's layout and in-place update (one launch per
// band, the window maximum as a scan over the window).  They are the simple
// reference-shaped path; the fused engine (engine.cu) is the fast one.
#include <climits>

#include "common.cuh"

namespace fhtdp {
namespace {

template <typename Acc>
__device__ __forceinline__ size_t cell(const Shape &s, int band, int x, int d) {
    int sign = d < 0 ? 1 : 0;
    int sh = d < 0 ? -d : d;
    return (((size_t)band * 2 + sign) * s.n + sh) * s.W + x;
}

template <typename Acc>
__device__ __forceinline__ Acc vmax(Acc a, Acc b) {
    return a > b ? a : b;
}

// Band k-1: V = H where the link ends inside the image, dead elsewhere.
template <typename Acc>
__global__ void dp_last_band_kernel(Acc *hv, Shape s) {
    const int band = s.k - 1;
    const size_t per_band = (size_t)2 * s.n * s.W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per_band;
         i += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(i % s.W);
        int r = (int)(i / s.W);
        int sh = r % s.n, sign = r / s.n;
        int d = sign ? -sh : sh;
        if (x >= s.w || x + d < 0 || x + d >= s.w)
            hv[(size_t)band * per_band + i] = Dead<Acc>::value();
    }
}

// Band `band` < k-1, given V of band+1 already in place.
template <typename Acc>
__global__ void dp_band_kernel(Acc *hv, Shape s, int band, int B) {
    const size_t per_band = (size_t)2 * s.n * s.W;
    const Acc dead = Dead<Acc>::value();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per_band;
         i += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(i % s.W);
        int r = (int)(i / s.W);
        int sh = r % s.n, sign = r / s.n;
        int d = sign ? -sh : sh;
        size_t idx = (size_t)band * per_band + i;
        int xn = x + d;
        if (x >= s.w || xn < 0 || xn >= s.w) {
            hv[idx] = dead;
            continue;
        }
        int lo = max(d - B, -(s.n - 1)), hi = min(d + B, s.n - 1);
        Acc best = dead;
        for (int e = lo; e <= hi; ++e) best = vmax(best, hv[cell<Acc>(s, band + 1, xn, e)]);
        hv[idx] = (best == dead) ? dead : hv[idx] + best;
    }
}

// One block: lexicographically smallest argmax of V_0, then the read-back.
template <typename Acc>
__global__ void backtrack_kernel(const Acc *V, Shape s, int B, int32_t *x_out, int32_t *d_out,
                                 Acc *score_out) {
    __shared__ Acc sv[1024];
    __shared__ int si[1024];
    const Acc dead = Dead<Acc>::value();
    Acc best = dead;
    int bidx = INT_MAX;
    const int total = s.w * s.D;   // lexicographic index x * D + (d + n - 1)
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int x = idx / s.D, d = idx % s.D - (s.n - 1);
        Acc v = V[cell<Acc>(s, 0, x, d)];
        if (v > best) {            // indices grow, so the first max is kept
            best = v;
            bidx = idx;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bidx;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            Acc ov = sv[threadIdx.x + off];
            int oi = si[threadIdx.x + off];
            if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                sv[threadIdx.x] = ov;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    int x = si[0] / s.D, d = si[0] % s.D - (s.n - 1);
    x_out[0] = x;
    d_out[0] = d;
    *score_out = sv[0];
    for (int i = 1; i < s.k; ++i) {
        x += d;
        int lo = max(d - B, -(s.n - 1)), hi = min(d + B, s.n - 1);
        Acc bv = dead;
        int be = lo;
        for (int e = lo; e <= hi; ++e) {
            Acc v = V[cell<Acc>(s, i, x, e)];
            if (v > bv) {
                bv = v;
                be = e;
            }
        }
        d = be;
        x_out[i] = x;
        d_out[i] = d;
    }
    x_out[s.k] = x + d;
}

int grid_for(size_t total) {
    size_t blocks = (total + 255) / 256;
    size_t cap = 152 * 16;
    return (int)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

}  // namespace

template <typename Acc>
int launch_dp_inplace(Acc *hv, const Shape &s, int B, cudaStream_t stream) {
    const size_t per_band = (size_t)2 * s.n * s.W;
    dp_last_band_kernel<Acc><<<grid_for(per_band), 256, 0, stream>>>(hv, s);
    int st = launched("dp_last_band_kernel");
    for (int band = s.k - 2; band >= 0 && !st; --band) {
        dp_band_kernel<Acc><<<grid_for(per_band), 256, 0, stream>>>(hv, s, band, B);
        st = launched("dp_band_kernel");
    }
    return st;
}

template <typename Acc>
int launch_backtrack(const Acc *V, const Shape &s, int B, int32_t *x_out, int32_t *d_out,
                     Acc *score_out, cudaStream_t stream) {
    backtrack_kernel<Acc><<<1, 1024, 0, stream>>>(V, s, B, x_out, d_out, score_out);
    return launched("backtrack_kernel");
}

template int launch_dp_inplace<int32_t>(int32_t *, const Shape &, int, cudaStream_t);
template int launch_dp_inplace<float>(float *, const Shape &, int, cudaStream_t);
template int launch_backtrack<int32_t>(const int32_t *, const Shape &, int, int32_t *, int32_t *,
                                       int32_t *, cudaStream_t);
template int launch_backtrack<float>(const float *, const Shape &, int, int32_t *, int32_t *,
                                     float *, cudaStream_t);

}  // namespace fhtdp
