// In-place DP over the Hough images and the read-back (the standalone
// fhtdp_polyline_dp / fhtdp_backtrack calls).
//
// Sec. 2.2-2.3, Eqs. 3-4: going up from the last band, every Hough cell
// (x, d) of band i is increased by the best admissible continuation in band
// i+1, i.e. the maximum of V_{i+1}(x + d, e) over the continuation window of
// d: the integer bend limit |e - d| <= B, or the bend-angle range of Eqs. 6-7
// (both as a window table).  Eq. 5 and the main problem's steps 2-3: the best
// top point is the maximum of V_0, and the polyline is read back band by band.
//
// These kernels keep the paper's layout and in-place update (one launch per
// band).  They are the modular path, the path of 256-row bands, of the main
// problem's angle windows and of the through-point query; the fused engine
// (engine.cu) is the fast one for integer bend limits and bands of up to 128
// rows.
#include <climits>
#include <functional>

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

// Continuation windows of the read-back: the integer bend limit |e - d| <= B,
// or the bend-angle table of the main problem.  B is clamped to 2n-2 (a wider
// limit admits nothing more), so d +/- B never overflows.
struct BendWin {
    int B, n;
    __host__ __device__ BendWin(int b, int nn) : B(b < 2 * nn - 2 ? b : 2 * nn - 2), n(nn) {}
    __device__ int lo(int d) const { return max(d - B, -(n - 1)); }
    __device__ int hi(int d) const { return min(d + B, n - 1); }
};
struct TableWin {
    WindowTable t;
    __device__ int lo(int d) const { return t.lo[d + t.n - 1]; }
    __device__ int hi(int d) const { return t.hi[d + t.n - 1]; }
};

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
        if (x >= s.vw || x + d < 0 || x + d >= s.vw)
            hv[(size_t)band * per_band + i] = Dead<Acc>::value();
    }
}


// The through-point restriction (Subproblems 2-3): every state of `band`
// whose vertex on the point's border is not xp becomes dead: the link's
// start x when the point is on the band's upper border, its end x + d when
// it is on the band's lower border (the image's bottom, end = 1).
template <typename Acc>
__global__ void point_mask_kernel(Acc *hv, Shape s, int band, int xp, int end) {
    const size_t per_band = (size_t)2 * s.n * s.W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per_band;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % s.W);
        const int r = (int)(i / s.W);
        const int sh = r % s.n, sign = r / s.n;
        const int d = sign ? -sh : sh;
        if ((end ? x + d : x) != xp) hv[(size_t)band * per_band + i] = Dead<Acc>::value();
    }
}

// Band `band` < k-1 of the DP, given V of band+1 already in place (Sec.
// 2.2-2.3, Eqs. 3-4, RangeMaxQ): V_b(x, d) = H_b(x, d) + max_{lo(d) <= e <=
// hi(d)} V_{b+1}(x + d, e), dead when x + d leaves the image or every e is
// dead.  The window table is the integer bend limit |e - d| <= B or the
// bend-angle range of Eqs. 6-7.  A block owns C continuation columns xn (the
// grid covers xn in [-(n-1), W + n - 1), so every state (x, d), x in [0, W),
// has exactly one owner xn = x + d).  The windows differ in length, so each
// one is answered as a range-maximum query on a sparse table kept whole in
// shared memory: level j holds, for every displacement, the maximum of the
// 2^j from it on, and a window of length L with 2^j <= L < 2^(j+1) is the
// maximum of the level-j runs starting at lo and at hi - 2^j + 1.  Max is
// exact, so the values are those of the scan over the window, and the one
// addition per state is the same as the oracle's.
//
// A thread owns column c = tid % C and rows r = tid / C + 32 u, u < RPT
// (32 * RPT >= 2n - 1): its window bounds and H_b values stay in registers,
// all its loads are issued before the first shared-memory store, and the
// results leave as plain stores (both copies of d = 0).  `levels` =
// floor(log2(longest window)) + 1.
template <typename Acc, int C, int RPT>
__global__ void __launch_bounds__(32 * C)
dp_band_window_kernel(Acc *hv, Shape s, int band, WindowTable t, int levels) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Acc *sm = (Acc *)smraw;
    const int D = s.D;
    const int c = threadIdx.x % C, r0 = threadIdx.x / C;
    const int xn0 = (int)blockIdx.x * C - (s.n - 1), xn = xn0 + c;
    const Acc dead = Dead<Acc>::value();
    const size_t dup_row = ((size_t)band * 2 + 1) * s.n * s.W;   // d = 0, "-" half
    if (!(xn0 + C > 0 && xn0 < s.vw)) {
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int r = r0 + 32 * u, d = r - (s.n - 1), x = xn - d;
            if (r >= D || x < 0 || x >= s.W) continue;
            hv[cell<Acc>(s, band, x, d)] = dead;
            if (d == 0) hv[dup_row + x] = dead;
        }
        return;
    }
    const bool live_col = xn >= 0 && xn < s.vw;
    Acc va[RPT], hb[RPT];
    uint32_t lh[RPT];   // window rows lo | hi << 16
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int r = r0 + 32 * u, d = r - (s.n - 1), x = xn - d;
        va[u] = dead;
        hb[u] = Acc(0);
        lh[u] = 0;
        if (r < D) {
            if (live_col) va[u] = hv[cell<Acc>(s, band + 1, xn, d)];
            if (live_col && x >= 0 && x < s.vw) hb[u] = hv[cell<Acc>(s, band, x, d)];
            lh[u] = (uint32_t)(t.lo[r] + s.n - 1) | (uint32_t)(t.hi[r] + s.n - 1) << 16;
        }
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int r = r0 + 32 * u;
        if (r < D) sm[r * C + c] = va[u];
    }
    for (int j = 1; j < levels; ++j) {
        __syncthreads();
        const int len = 1 << (j - 1);
        const Acc *src = sm + (size_t)(j - 1) * D * C;
        Acc *dst = sm + (size_t)j * D * C;
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int r = r0 + 32 * u;
            if (r < D) dst[r * C + c] = r + len < D ? vmax(src[r * C + c], src[(r + len) * C + c])
                                                    : src[r * C + c];
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int r = r0 + 32 * u, d = r - (s.n - 1), x = xn - d;
        if (r >= D || x < 0 || x >= s.W) continue;
        Acc v = dead;
        if (x < s.vw && live_col) {
            const int lo = (int)(lh[u] & 0xffffu), hi = (int)(lh[u] >> 16);
            const int j = 31 - __clz(hi - lo + 1);
            const Acc *T = sm + (size_t)j * D * C;
            const Acc best = vmax(T[lo * C + c], T[(hi - (1 << j) + 1) * C + c]);
            v = (best == dead) ? dead : hb[u] + best;
        }
        hv[cell<Acc>(s, band, x, d)] = v;
        if (d == 0) hv[dup_row + x] = v;
    }
}

// Order-preserving 32-bit image of a value (negative zero counts as zero).
__device__ __forceinline__ uint32_t vord(int32_t v) { return (uint32_t)v ^ 0x80000000u; }
__device__ __forceinline__ uint32_t vord(float f) {
    const uint32_t b = __float_as_uint(f == 0.0f ? 0.0f : f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
template <typename Acc>
__device__ __forceinline__ Acc vfrom(uint32_t o);
template <>
__device__ __forceinline__ int32_t vfrom<int32_t>(uint32_t o) {
    return (int32_t)(o ^ 0x80000000u);
}
template <>
__device__ __forceinline__ float vfrom<float>(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Grid-wide argmax of V_0 as one 64-bit key: the value's order image above
// the complement of the lexicographic index x * D + (d + n - 1), so that the
// largest key is the largest value at the smallest index (*key starts at 0).
template <typename Acc>
__global__ void argmax_kernel(const Acc *V, Shape s, unsigned long long *key) {
    const Acc dead = Dead<Acc>::value();
    unsigned long long best = 0;
    const int total = s.vw * s.D;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i / s.vw, x = i - e * s.vw;   // x fastest: coalesced rows
        const Acc v = V[cell<Acc>(s, 0, x, e - (s.n - 1))];
        if (v == dead) continue;
        const unsigned long long k = ((unsigned long long)vord(v) << 32) |
                                     (0xffffffffu - (unsigned)(x * s.D + e));
        best = best > k ? best : k;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = best > other ? best : other;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(key, best);
}

// The second of two different extreme polylines: as argmax_kernel over the
// columns x with |x - x_0| >= sep, x_0 the top vertex of the optimum in key1.
template <typename Acc>
__global__ void argmax_apart_kernel(const Acc *V, Shape s, const unsigned long long *key1,
                                    int sep, unsigned long long *key2) {
    const unsigned long long k1 = *key1;
    if (k1 == 0) return;
    const int x0 = (int)((0xffffffffu - (unsigned)(k1 & 0xffffffffu)) / s.D);
    unsigned long long best = 0;
    const int total = s.vw * s.D;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i / s.vw, x = i - e * s.vw;
        if (abs(x - x0) < sep) continue;
        const Acc v = V[cell<Acc>(s, 0, x, e - (s.n - 1))];
        if (v == Dead<Acc>::value()) continue;
        const unsigned long long k = ((unsigned long long)vord(v) << 32) |
                                     (0xffffffffu - (unsigned)(x * s.D + e));
        best = best > k ? best : k;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = best > other ? best : other;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(key2, best);
}

// One warp: the read-back from the argmax key (Eq. 5); every band's window
// is scanned by the lanes, the first maximum kept.  No admissible state
// (key 0): x = -1 everywhere and a dead score.
template <typename Acc, typename Win>
__global__ void readback_kernel(const Acc *V, Shape s, Win win, const unsigned long long *key,
                                int32_t *x_out, int32_t *d_out, Acc *score_out) {
    const int lane = threadIdx.x;
    const Acc dead = Dead<Acc>::value();
    const unsigned long long kv = *key;
    if (kv == 0) {
        if (lane == 0) {
            *score_out = dead;
            for (int i = 0; i <= s.k; ++i) x_out[i] = -1;
            for (int i = 0; i < s.k; ++i) d_out[i] = 0;
        }
        return;
    }
    const unsigned lin = 0xffffffffu - (unsigned)(kv & 0xffffffffu);
    int x = (int)(lin / s.D), d = (int)(lin % s.D) - (s.n - 1);
    if (lane == 0) {
        x_out[0] = x;
        d_out[0] = d;
        *score_out = vfrom<Acc>((uint32_t)(kv >> 32));
    }
    for (int i = 1; i < s.k; ++i) {
        x += d;
        const int lo = win.lo(d), hi = win.hi(d);
        Acc bv = dead;
        int be = INT_MAX;
        for (int e = lo + lane; e <= hi; e += 32) {
            const Acc v = V[cell<Acc>(s, i, x, e)];
            if (v > bv) {
                bv = v;
                be = e;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const Acc ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oe = __shfl_xor_sync(0xffffffffu, be, o);
            if (ov > bv || (ov == bv && oe < be)) {
                bv = ov;
                be = oe;
            }
        }
        d = be == INT_MAX ? lo : be;
        if (lane == 0) {
            x_out[i] = x;
            d_out[i] = d;
        }
    }
    if (lane == 0) x_out[s.k] = x + d;
}

// One block: lexicographically smallest argmax of V_0, then the read-back.
template <typename Acc, typename Win>
__global__ void backtrack_kernel(const Acc *V, Shape s, Win win, int32_t *x_out, int32_t *d_out,
                                 Acc *score_out) {
    __shared__ Acc sv[1024];
    __shared__ int si[1024];
    const Acc dead = Dead<Acc>::value();
    Acc best = dead;
    int bidx = INT_MAX;
    const int total = s.vw * s.D;   // lexicographic index x * D + (d + n - 1)
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
        int lo = win.lo(d), hi = win.hi(d);
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
int launch_dp_inplace(Acc *hv, const Shape &s, int B, cudaStream_t stream, const PointMask *pm) {
    WindowTable t;
    make_bend_table(s.n, B, &t);
    return launch_dp_window<Acc>(hv, s, t, stream, pm);
}

template <typename Acc>
int launch_backtrack(const Acc *V, const Shape &s, int B, int32_t *x_out, int32_t *d_out,
                     Acc *score_out, cudaStream_t stream) {
    backtrack_kernel<Acc, BendWin><<<1, 1024, 0, stream>>>(V, s, BendWin{B, s.n}, x_out, d_out,
                                                            score_out);
    return launched("backtrack_kernel");
}

template <typename Acc>
int launch_backtrack_key(const Acc *V, const Shape &s, int B, unsigned long long *key,
                         int32_t *x_out, int32_t *d_out, Acc *score_out, cudaStream_t stream) {
    argmax_kernel<Acc><<<grid_for((size_t)s.vw * s.D), 256, 0, stream>>>(V, s, key);
    int st = launched("argmax_kernel");
    if (st) return st;
    readback_kernel<Acc, BendWin><<<1, 32, 0, stream>>>(V, s, BendWin{B, s.n}, key, x_out, d_out,
                                                         score_out);
    return launched("readback_kernel");
}

void make_bend_table(int n, int B, WindowTable *t) {
    const int D = 2 * n - 1;
    if (B > D - 1) B = D - 1;   // a wider limit admits nothing more (and 2B + 1 cannot overflow)
    for (int i = 0; i < kMaxD; ++i) {
        const int d = i - (n - 1);
        t->lo[i] = (int16_t)(i < D ? (d - B > -(n - 1) ? d - B : -(n - 1)) : 0);
        t->hi[i] = (int16_t)(i < D ? (d + B < n - 1 ? d + B : n - 1) : 0);
    }
    t->n = n;
    t->maxlen = 2 * B + 1 < D ? 2 * B + 1 : D;
}

namespace {
template <typename Acc, int C, int RPT>
int launch_dp_window_tiles(Acc *hv, const Shape &s, const WindowTable &t, cudaStream_t stream,
                           const std::function<int(int)> &after_band) {
    int levels = 1;
    while ((2 << (levels - 1)) <= t.maxlen) ++levels;   // floor(log2(maxlen)) + 1
    const size_t smem = (size_t)levels * s.D * C * sizeof(Acc);   // <= 9 * 511 * 8 * 4 = 147 KB
    static int smem_set = 48 * 1024;   // dynamic shared memory enabled so far
    if ((int)smem > smem_set) {
        int st = cuda_status(cudaFuncSetAttribute(dp_band_window_kernel<Acc, C, RPT>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)smem),
                             "cudaFuncSetAttribute");
        if (st) return st;
        smem_set = (int)smem;
    }
    const int blocks = (s.W + 2 * (s.n - 1) + C - 1) / C;
    int st = FHTDP_OK;
    for (int band = s.k - 2; band >= 0 && !st; --band) {
        dp_band_window_kernel<Acc, C, RPT><<<blocks, 32 * C, smem, stream>>>(hv, s, band, t,
                                                                             levels);
        st = launched("dp_band_window_kernel");
        if (!st) st = after_band(band);
    }
    return st;
}
}  // namespace

template <typename Acc>
int launch_dp_window(Acc *hv, const Shape &s, const WindowTable &t, cudaStream_t stream,
                     const PointMask *pm) {
    const size_t per_band = (size_t)2 * s.n * s.W;
    // The point's band: j (its upper border), or k-1 for the image's bottom
    // border, masked right after the band is formed.
    const std::function<int(int)> mask = [&](int band) -> int {
        if (!pm || band != (pm->j < s.k ? pm->j : s.k - 1)) return FHTDP_OK;
        point_mask_kernel<Acc><<<grid_for(per_band), 256, 0, stream>>>(hv, s, band, pm->xp,
                                                                       pm->j == s.k ? 1 : 0);
        return launched("point_mask_kernel");
    };
    dp_last_band_kernel<Acc><<<grid_for(per_band), 256, 0, stream>>>(hv, s);
    int st = launched("dp_last_band_kernel");
    if (!st) st = mask(s.k - 1);
    if (st || s.k == 1) return st;
    // 16 continuation columns per block (64-byte row segments) while that
    // still gives two blocks per SM, else 8; 32 * RPT >= 2n - 1 rows.
    const int span = s.W + 2 * (s.n - 1);
    const bool wide = (span + 15) / 16 >= 2 * 152 && s.D <= 32 * 8;
    if (s.D <= 32 * 4)
        return wide ? launch_dp_window_tiles<Acc, 16, 4>(hv, s, t, stream, mask)
                    : launch_dp_window_tiles<Acc, 8, 4>(hv, s, t, stream, mask);
    if (s.D <= 32 * 8)
        return wide ? launch_dp_window_tiles<Acc, 16, 8>(hv, s, t, stream, mask)
                    : launch_dp_window_tiles<Acc, 8, 8>(hv, s, t, stream, mask);
    return launch_dp_window_tiles<Acc, 8, 16>(hv, s, t, stream, mask);   // 256-row bands
}

template <typename Acc>
int launch_argmax_apart(const Acc *V, const Shape &s, const unsigned long long *key1, int sep,
                        unsigned long long *key2, cudaStream_t stream) {
    argmax_apart_kernel<Acc><<<grid_for((size_t)s.vw * s.D), 256, 0, stream>>>(V, s, key1, sep,
                                                                                key2);
    return launched("argmax_apart_kernel");
}

template <typename Acc>
int launch_readback_key(const Acc *V, const Shape &s, int B, const unsigned long long *key,
                        int32_t *x_out, int32_t *d_out, Acc *score_out, cudaStream_t stream) {
    readback_kernel<Acc, BendWin><<<1, 32, 0, stream>>>(V, s, BendWin{B, s.n}, key, x_out, d_out,
                                                         score_out);
    return launched("readback_kernel");
}

template <typename Acc>
int launch_backtrack_angle_key(const Acc *V, const Shape &s, const WindowTable &t,
                               unsigned long long *key, int32_t *x_out, int32_t *d_out,
                               Acc *score_out, cudaStream_t stream) {
    argmax_kernel<Acc><<<grid_for((size_t)s.vw * s.D), 256, 0, stream>>>(V, s, key);
    int st = launched("argmax_kernel");
    if (st) return st;
    readback_kernel<Acc, TableWin><<<1, 32, 0, stream>>>(V, s, TableWin{t}, key, x_out, d_out,
                                                         score_out);
    return launched("readback_kernel");
}

template <typename Acc>
int launch_backtrack_angle(const Acc *V, const Shape &s, const WindowTable &t, int32_t *x_out,
                           int32_t *d_out, Acc *score_out, cudaStream_t stream) {
    backtrack_kernel<Acc, TableWin><<<1, 1024, 0, stream>>>(V, s, TableWin{t}, x_out, d_out,
                                                            score_out);
    return launched("backtrack_kernel");
}

#define FHTDP_INSTANTIATE_QUERIES(Acc)                                                          \
    template int launch_argmax_apart<Acc>(const Acc *, const Shape &,                           \
                                          const unsigned long long *, int,                      \
                                          unsigned long long *, cudaStream_t);                  \
    template int launch_readback_key<Acc>(const Acc *, const Shape &, int,                      \
                                          const unsigned long long *, int32_t *, int32_t *,     \
                                          Acc *, cudaStream_t);                                 \
    template int launch_backtrack_angle_key<Acc>(const Acc *, const Shape &,                    \
                                                 const WindowTable &, unsigned long long *,     \
                                                 int32_t *, int32_t *, Acc *, cudaStream_t);    \
    template int launch_backtrack_angle<Acc>(const Acc *, const Shape &, const WindowTable &,   \
                                             int32_t *, int32_t *, Acc *, cudaStream_t);
FHTDP_INSTANTIATE_QUERIES(int32_t)
FHTDP_INSTANTIATE_QUERIES(float)
#undef FHTDP_INSTANTIATE_QUERIES

template int launch_dp_window<int32_t>(int32_t *, const Shape &, const WindowTable &,
                                       cudaStream_t, const PointMask *);
template int launch_dp_window<float>(float *, const Shape &, const WindowTable &, cudaStream_t,
                                     const PointMask *);
template int launch_dp_inplace<int32_t>(int32_t *, const Shape &, int, cudaStream_t,
                                        const PointMask *);
template int launch_dp_inplace<float>(float *, const Shape &, int, cudaStream_t,
                                      const PointMask *);
template int launch_backtrack_key<int32_t>(const int32_t *, const Shape &, int,
                                           unsigned long long *, int32_t *, int32_t *, int32_t *,
                                           cudaStream_t);
template int launch_backtrack_key<float>(const float *, const Shape &, int, unsigned long long *,
                                         int32_t *, int32_t *, float *, cudaStream_t);
template int launch_backtrack<int32_t>(const int32_t *, const Shape &, int, int32_t *, int32_t *,
                                       int32_t *, cudaStream_t);
template int launch_backtrack<float>(const float *, const Shape &, int, int32_t *, int32_t *,
                                     float *, cudaStream_t);

}  // namespace fhtdp
