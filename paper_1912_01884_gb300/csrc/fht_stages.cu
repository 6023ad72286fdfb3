// Band FHT, one dyadic level per launch (the standalone fhtdp_fht_bands).
//
// Sec. 2.1 (refs [10], [34]): the Hough image of a band is built bottom-up
// over sub-bands of 1, 2, 4, ..., n rows.  Merging the top half A and the
// bottom half B of a sub-band of m rows gives, for every shift s in [0, m),
//   out(x, s) = A(x, s>>1) + B(x +/- ceil(s/2), s>>1)      (columns mod W)
// with "+" for lines moving right and "-" for lines moving left.  The sum
// tree is therefore fixed (top half + bottom half at every level), which
// makes the float path reproducible bit for bit.
//
// Layout of every level: [band][sign][row][x], x fastest; at the level of
// m-row sub-bands, row j*m + s holds shift s of sub-band j, so the last level
// (m = n, one sub-band) is exactly the [k][2][n][W] Hough layout.
// Each level is a coalesced streaming pass: a warp reads a contiguous row
// segment of A and a contiguous (shifted) segment of B.
#include "common.cuh"

namespace fhtdp {
namespace {

template <typename In, typename Acc>
__device__ __forceinline__ Acc band_pixel(const In *img, int pitch, int w, int row, int col) {
    return col < w ? static_cast<Acc>(img[(size_t)row * pitch + col]) : Acc(0);
}

__device__ __forceinline__ int wrap(int x, int W) {
    return x >= W ? x - W : (x < 0 ? x + W : x);
}

// n == 1: the band is a single row, and both "signs" are the padded row.
template <typename In, typename Acc>
__global__ void fht_single_row_kernel(const In *img, int pitch, Shape s, Acc *out) {
    const size_t total = (size_t)s.k * 2 * s.W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(i % s.W);
        int band = (int)(i / s.W) / 2;
        out[i] = band_pixel<In, Acc>(img, pitch, s.w, band, x);
    }
}

// Level of 2-row sub-bands, read straight from the image (zero padding is
// the predicate col < w, never stored).
template <typename In, typename Acc>
__global__ void fht_level2_kernel(const In *img, int pitch, Shape s, Acc *out) {
    const size_t total = (size_t)s.k * 2 * s.n * s.W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(i % s.W);
        size_t r = i / s.W;
        int row = (int)(r % s.n);
        int bs = (int)(r / s.n);
        int sign = bs & 1, band = bs >> 1;
        int sh = row & 1;                       // shift within the 2-row sub-band
        int ya = band * s.n + (row & ~1);       // top row of the sub-band
        int xb = wrap(sign == 0 ? x + sh : x - sh, s.W);
        out[i] = band_pixel<In, Acc>(img, pitch, s.w, ya, x) +
                 band_pixel<In, Acc>(img, pitch, s.w, ya + 1, xb);
    }
}

// Level of m-row sub-bands (m >= 4) from the level of m/2-row sub-bands.
template <typename Acc>
__global__ void fht_level_kernel(const Acc *__restrict__ src, Shape s, int m,
                                 Acc *__restrict__ dst) {
    const size_t total = (size_t)s.k * 2 * s.n * s.W;
    const int half = m >> 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(i % s.W);
        size_t r = i / s.W;
        int row = (int)(r % s.n);
        size_t bs = r / s.n;
        int sign = (int)(bs & 1);
        int j0 = row & ~(m - 1);                // first row of the sub-band
        int sh = row & (m - 1);                 // shift in [0, m)
        int move = sh - (sh >> 1);              // ceil(sh / 2)
        int xb = wrap(sign == 0 ? x + move : x - move, s.W);
        const Acc *base = src + bs * s.n * (size_t)s.W;
        Acc a = base[(size_t)(j0 + (sh >> 1)) * s.W + x];
        Acc b = base[(size_t)(j0 + half + (sh >> 1)) * s.W + xb];
        dst[i] = a + b;
    }
}

// Two levels in one pass: sub-bands of M = 4m rows from the level of m-row
// sub-bands J0..J3.  With S the shift, s2 = S >> 1 and q = S >> 2,
//   out(x, S) = [J0(x, q) + J1(x +/- ceil(s2/2), q)]
//             + [J2(x', q) + J3(x' +/- ceil(s2/2), q)],   x' = x +/- ceil(S/2),
// the same sum tree as the two radix-2 levels (so float sums are unchanged).
template <typename Acc>
__global__ void fht_level4_kernel(const Acc *__restrict__ src, Shape s, int M,
                                  Acc *__restrict__ dst) {
    const size_t total = (size_t)s.k * 2 * s.n * s.W;
    const int m = M >> 2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % s.W);
        const size_t r = i / s.W;
        const int row = (int)(r % s.n);
        const size_t bs = r / s.n;
        const int sign = (int)(bs & 1);
        const int j0 = row & ~(M - 1);
        const int S = row & (M - 1), s2 = S >> 1, q = S >> 2;
        const int c2 = s2 - (s2 >> 1), cS = S - (S >> 1);
        const int x1 = wrap(sign == 0 ? x + c2 : x - c2, s.W);
        const int xp = wrap(sign == 0 ? x + cS : x - cS, s.W);
        const int x3 = wrap(sign == 0 ? xp + c2 : xp - c2, s.W);
        const Acc *base = src + bs * s.n * (size_t)s.W;
        const Acc a0 = base[(size_t)(j0 + q) * s.W + x];
        const Acc a1 = base[(size_t)(j0 + m + q) * s.W + x1];
        const Acc a2 = base[(size_t)(j0 + 2 * m + q) * s.W + xp];
        const Acc a3 = base[(size_t)(j0 + 3 * m + q) * s.W + x3];
        dst[i] = (a0 + a1) + (a2 + a3);
    }
}

int grid_for(size_t total) {
    size_t blocks = (total + 255) / 256;
    size_t cap = 152 * 16;
    return (int)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

// Binomial weights C(2r, r + t), |t| <= r, by value.
struct GaussWeights {
    int32_t c[2 * kMaxGaussR + 1];
};

constexpr int kGaussSeg = 1024;   // output columns per block (4 per thread)

// Main problem, step 1 (Sec. 2.3): every row convolved with the discrete
// Gaussian of half-width r, the unnormalised binomial weights (integer
// arithmetic, so the sums are exact); pixels outside the row count as zero.
// A block stages one row segment and its 2r-pixel halo in shared memory as
// int32 and writes kGaussSeg outputs of the dense [h][w] result.
template <typename In>
__global__ void gauss_rows_kernel(const In *__restrict__ img, int pitch, int w, int r,
                                  GaussWeights g, int32_t *__restrict__ out) {
    __shared__ int32_t seg[kGaussSeg + 2 * kMaxGaussR];
    const int y = blockIdx.x;
    const int x0 = blockIdx.y * kGaussSeg;
    const In *row = img + (size_t)y * pitch;
    for (int i = threadIdx.x; i < kGaussSeg + 2 * r; i += blockDim.x) {
        const int c = x0 - r + i;
        seg[i] = (c >= 0 && c < w) ? (int32_t)row[c] : 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kGaussSeg; i += blockDim.x) {
        const int x = x0 + i;
        if (x >= w) break;
        int32_t acc = 0;
        for (int t = 0; t <= 2 * r; ++t) acc += g.c[t] * seg[i + t];
        out[(size_t)y * w + x] = acc;
    }
}

}  // namespace

template <typename In>
int launch_gauss_rows(const In *img, int pitch, int h, int w, int r, int32_t *out,
                      cudaStream_t stream) {
    GaussWeights g{};
    g.c[0] = 1;
    for (int j = 1; j <= 2 * r; ++j)   // row 2r of Pascal's triangle
        g.c[j] = (int32_t)((int64_t)g.c[j - 1] * (2 * r - j + 1) / j);
    dim3 grid((unsigned)h, (unsigned)((w + kGaussSeg - 1) / kGaussSeg));   // rows in x: h <= 2^20
    gauss_rows_kernel<In><<<grid, 256, 0, stream>>>(img, pitch, w, r, g, out);
    return launched("gauss_rows_kernel");
}

template int launch_gauss_rows<uint8_t>(const uint8_t *, int, int, int, int, int32_t *,
                                        cudaStream_t);
template int launch_gauss_rows<int32_t>(const int32_t *, int, int, int, int, int32_t *,
                                        cudaStream_t);

template <typename In, typename Acc>
int launch_fht_stages(const In *img, int pitch, const Shape &s, Acc *hough, Acc *tmp,
                      cudaStream_t stream) {
    if (s.n == 1) {
        size_t total = (size_t)s.k * 2 * s.W;
        fht_single_row_kernel<In, Acc><<<grid_for(total), 256, 0, stream>>>(img, pitch, s, hough);
        return launched("fht_single_row_kernel");
    }
    const size_t total = (size_t)s.k * 2 * s.n * s.W;
    const int levels = s.log2n;
    // Passes: level 1 from the image, then two levels at a time, then one
    // if a level is left.  The passes alternate between tmp and hough so
    // that the last one lands in hough.
    const int passes = 1 + (levels - 1) / 2 + (levels - 1) % 2;
    int pass = 0;
    auto dst_of = [&](int p) { return ((passes - 1 - p) % 2 == 0) ? hough : tmp; };
    fht_level2_kernel<In, Acc><<<grid_for(total), 256, 0, stream>>>(img, pitch, s, dst_of(0));
    int st = launched("fht_level2_kernel");
    int l = 1;
    for (; l + 2 <= levels && !st; l += 2, ++pass) {
        fht_level4_kernel<Acc><<<grid_for(total), 256, 0, stream>>>(dst_of(pass), s, 1 << (l + 2),
                                                                    dst_of(pass + 1));
        st = launched("fht_level4_kernel");
    }
    if (l < levels && !st) {
        fht_level_kernel<Acc><<<grid_for(total), 256, 0, stream>>>(dst_of(pass), s, 1 << levels,
                                                                   dst_of(pass + 1));
        st = launched("fht_level_kernel");
    }
    return st;
}

template int launch_fht_stages<uint8_t, int32_t>(const uint8_t *, int, const Shape &, int32_t *,
                                                 int32_t *, cudaStream_t);
template int launch_fht_stages<int32_t, int32_t>(const int32_t *, int, const Shape &, int32_t *,
                                                 int32_t *, cudaStream_t);
template int launch_fht_stages<float, float>(const float *, int, const Shape &, float *, float *,
                                             cudaStream_t);

}  // namespace fhtdp
