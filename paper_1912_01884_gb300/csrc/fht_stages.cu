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

// Every pass below gives one block one row of its output level ([band]
// [sign][row], blockIdx.x, up to 2h rows) and its threads the columns, so the
// row's shifts are computed once and each column costs only its loads.

// Level of 2-row sub-bands, read straight from the image (zero padding is
// the predicate col < w, never stored).
template <typename In, typename Acc>
__global__ void fht_level2_kernel(const In *img, int pitch, Shape s, Acc *out) {
    const int r = blockIdx.x;
    const int row = r % s.n, bs = r / s.n;
    const int sign = bs & 1, band = bs >> 1;
    const int sh = row & 1;                     // shift within the 2-row sub-band
    const int ya = band * s.n + (row & ~1);     // top row of the sub-band
    Acc *dst = out + (size_t)r * s.W;
    for (int x = threadIdx.x; x < s.W; x += blockDim.x) {
        const int xb = wrap(sign == 0 ? x + sh : x - sh, s.W);
        dst[x] = band_pixel<In, Acc>(img, pitch, s.w, ya, x) +
                 band_pixel<In, Acc>(img, pitch, s.w, ya + 1, xb);
    }
}

// Level of m-row sub-bands (m >= 4) from the level of m/2-row sub-bands.
template <typename Acc>
__global__ void fht_level_kernel(const Acc *__restrict__ src, Shape s, int m,
                                 Acc *__restrict__ dst) {
    const int r = blockIdx.x;
    const int row = r % s.n, bs = r / s.n;
    const int sign = bs & 1;
    const int j0 = row & ~(m - 1);              // first row of the sub-band
    const int sh = row & (m - 1);               // shift in [0, m)
    const int move = sh - (sh >> 1);            // ceil(sh / 2)
    const Acc *base = src + (size_t)bs * s.n * s.W;
    const Acc *ra = base + (size_t)(j0 + (sh >> 1)) * s.W;
    const Acc *rb = base + (size_t)(j0 + (m >> 1) + (sh >> 1)) * s.W;
    Acc *out = dst + (size_t)r * s.W;
#pragma unroll 4
    for (int x = threadIdx.x; x < s.W; x += blockDim.x) {
        const int xb = wrap(sign == 0 ? x + move : x - move, s.W);
        out[x] = ra[x] + rb[xb];
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
    const int m = M >> 2;
    const int r = blockIdx.x;
    const int row = r % s.n, bs = r / s.n;
    const int sign = bs & 1;
    const int j0 = row & ~(M - 1);
    const int S = row & (M - 1), s2 = S >> 1, q = S >> 2;
    const int c2 = s2 - (s2 >> 1), cS = S - (S >> 1);
    const Acc *base = src + (size_t)bs * s.n * s.W;
    const Acc *r0 = base + (size_t)(j0 + q) * s.W;
    const Acc *r1 = base + (size_t)(j0 + m + q) * s.W;
    const Acc *r2 = base + (size_t)(j0 + 2 * m + q) * s.W;
    const Acc *r3 = base + (size_t)(j0 + 3 * m + q) * s.W;
    Acc *out = dst + (size_t)r * s.W;
#pragma unroll 4
    for (int x = threadIdx.x; x < s.W; x += blockDim.x) {
        const int x1 = wrap(sign == 0 ? x + c2 : x - c2, s.W);
        const int xp = wrap(sign == 0 ? x + cS : x - cS, s.W);
        const int x3 = wrap(sign == 0 ? xp + c2 : xp - c2, s.W);
        out[x] = (r0[x] + r1[x1]) + (r2[xp] + r3[x3]);
    }
}

// Binomial weights C(2r, r + t), |t| <= r, by value.
struct GaussWeights {
    int32_t c[2 * kMaxGaussR + 1];
};

GaussWeights binomial_weights(int r) {
    GaussWeights g{};
    g.c[0] = 1;
    for (int j = 1; j <= 2 * r; ++j)   // row 2r of Pascal's triangle
        g.c[j] = (int32_t)((int64_t)g.c[j - 1] * (2 * r - j + 1) / j);
    return g;
}

// Pixel c of an image row after the row smoothing (zero in the padding
// columns c >= w and outside the row).  Acc = int32_t: exact integer sums;
// Acc = float: each product weight * pixel rounded, then added in the order
// t = -r .. r to an accumulator starting at 0 (the float32 reading of the
// smoothing step).
template <typename In, typename Acc>
__device__ __forceinline__ Acc smoothed(const In *row, int w, int r, const GaussWeights &g,
                                        int c) {
    if (c >= w) return Acc(0);
    Acc acc = 0;
    for (int t = -r; t <= r; ++t) {
        const int cc = c + t;
        if (cc >= 0 && cc < w) acc += (Acc)g.c[t + r] * (Acc)row[cc];
    }
    return acc;
}

constexpr int kL2Chunk = 1024;   // columns per block of the smoothing level-2 pass

// Main problem, step 1 fused into the first FHT level: a block takes one
// pair of image rows (the 2-row sub-band j of a band) and kL2Chunk columns.
// It stages both raw rows over the chunk and its halo (1 + r columns each
// side, zero outside the image) in shared memory, smooths the top row A at x
// and the bottom row B at x-1..x+chunk (columns mod W; a column that wraps
// around is smoothed from global memory), and writes the four level-2 rows
// of the pair: shifts 0 and 1 of both signs, A(x) + B(x) and A(x) + B(x +/- 1).
template <typename In, typename Acc>
__global__ void fht_level2_gauss_kernel(const In *img, int pitch, Shape s, int r,
                                        GaussWeights g, Acc *out) {
    constexpr int kRaw = kL2Chunk + 2 + 2 * kMaxGaussR;
    __shared__ Acc rawa[kRaw], rawb[kRaw], sa[kL2Chunk], sb[kL2Chunk + 2];
    const int half = s.n >> 1;
    const int pair = blockIdx.x;
    const int band = pair / half, j = pair - band * half;
    const int ya = band * s.n + 2 * j;
    const int x0 = blockIdx.y * kL2Chunk;
    const int cols = min(kL2Chunk, s.W - x0);
    const int base = x0 - 1 - r;   // image column of rawa[0] / rawb[0]
    const In *ra = img + (size_t)ya * pitch, *rb = ra + pitch;
    for (int i = threadIdx.x; i < cols + 2 + 2 * r; i += blockDim.x) {
        const int c = base + i;
        const bool in = c >= 0 && c < s.w;
        rawa[i] = in ? (Acc)ra[c] : Acc(0);
        rawb[i] = in ? (Acc)rb[c] : Acc(0);
    }
    __syncthreads();
    // Pixels outside the row add a zero product, which leaves an integer or
    // float sum unchanged (a float sum that starts at +0 never holds -0).
    for (int i = threadIdx.x; i < cols + 2; i += blockDim.x) {
        const int c = x0 - 1 + i, cw = wrap(c, s.W);
        Acc vb = 0;
        if (cw != c) {
            vb = smoothed<In, Acc>(rb, s.w, r, g, cw);
        } else if (c < s.w) {
            for (int t = 0; t <= 2 * r; ++t) vb += (Acc)g.c[t] * rawb[i + t];
        }
        sb[i] = vb;
        if (i < cols && c + 1 < s.w) {
            Acc va = 0;
            for (int t = 0; t <= 2 * r; ++t) va += (Acc)g.c[t] * rawa[i + 1 + t];
            sa[i] = va;
        } else if (i < cols) {
            sa[i] = 0;
        }
    }
    __syncthreads();
    Acc *plus = out + ((size_t)(band * 2) * s.n + 2 * j) * s.W;
    Acc *minus = out + ((size_t)(band * 2 + 1) * s.n + 2 * j) * s.W;
    for (int i = threadIdx.x; i < cols; i += blockDim.x) {
        const int x = x0 + i;
        const Acc A = sa[i], B = sb[i + 1];
        plus[x] = A + B;
        plus[s.W + x] = A + sb[i + 2];
        minus[x] = A + B;
        minus[s.W + x] = A + sb[i];
    }
}

int grid_for(size_t total) {
    size_t blocks = (total + 255) / 256;
    size_t cap = 152 * 16;
    return (int)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

constexpr int kGaussSeg = 1024;   // output columns per block (4 per thread)

// Main problem, step 1 (Sec. 2.3): every row convolved with the discrete
// Gaussian of half-width r, the unnormalised binomial weights (integer
// arithmetic for integer images, so the sums are exact; float images in the
// float order of `smoothed`); pixels outside the row count as zero.  A block
// stages one row segment and its 2r-pixel halo in shared memory and writes
// kGaussSeg outputs of the dense [h][w] result.
template <typename In, typename Acc>
__global__ void gauss_rows_kernel(const In *__restrict__ img, int pitch, int w, int r,
                                  GaussWeights g, Acc *__restrict__ out) {
    __shared__ Acc seg[kGaussSeg + 2 * kMaxGaussR];
    const int y = blockIdx.x;
    const int x0 = blockIdx.y * kGaussSeg;
    const In *row = img + (size_t)y * pitch;
    for (int i = threadIdx.x; i < kGaussSeg + 2 * r; i += blockDim.x) {
        const int c = x0 - r + i;
        seg[i] = (c >= 0 && c < w) ? (Acc)row[c] : Acc(0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kGaussSeg; i += blockDim.x) {
        const int x = x0 + i;
        if (x >= w) break;
        Acc acc = 0;
        for (int t = 0; t <= 2 * r; ++t) acc += (Acc)g.c[t] * seg[i + t];
        out[(size_t)y * w + x] = acc;
    }
}

}  // namespace

template <typename In, typename Acc>
int launch_gauss_rows(const In *img, int pitch, int h, int w, int r, Acc *out,
                      cudaStream_t stream) {
    const GaussWeights g = binomial_weights(r);
    dim3 grid((unsigned)h, (unsigned)((w + kGaussSeg - 1) / kGaussSeg));   // rows in x: h <= 2^20
    gauss_rows_kernel<In, Acc><<<grid, 256, 0, stream>>>(img, pitch, w, r, g, out);
    return launched("gauss_rows_kernel");
}

template int launch_gauss_rows<uint8_t, int32_t>(const uint8_t *, int, int, int, int, int32_t *,
                                                 cudaStream_t);
template int launch_gauss_rows<int32_t, int32_t>(const int32_t *, int, int, int, int, int32_t *,
                                                 cudaStream_t);
template int launch_gauss_rows<float, float>(const float *, int, int, int, int, float *,
                                             cudaStream_t);

namespace {
// The passes after level 2 (which the caller wrote into pass_dst(s, 0, ...)):
// two levels at a time, then one if a level is left.  The passes alternate
// between tmp and hough so that the last one lands in hough.
int fht_passes(const Shape &s) {
    const int levels = s.log2n;
    return 1 + (levels - 1) / 2 + (levels - 1) % 2;
}
template <typename Acc>
Acc *pass_dst(const Shape &s, int p, Acc *hough, Acc *tmp) {
    return ((fht_passes(s) - 1 - p) % 2 == 0) ? hough : tmp;
}
template <typename Acc>
int fht_upper_levels(const Shape &s, Acc *hough, Acc *tmp, cudaStream_t stream) {
    const int rows = s.k * 2 * s.n;
    const int levels = s.log2n;
    int st = FHTDP_OK, pass = 0, l = 1;
    for (; l + 2 <= levels && !st; l += 2, ++pass) {
        fht_level4_kernel<Acc><<<rows, 256, 0, stream>>>(pass_dst(s, pass, hough, tmp), s,
                                                          1 << (l + 2),
                                                          pass_dst(s, pass + 1, hough, tmp));
        st = launched("fht_level4_kernel");
    }
    if (l < levels && !st) {
        fht_level_kernel<Acc><<<rows, 256, 0, stream>>>(pass_dst(s, pass, hough, tmp), s,
                                                         1 << levels,
                                                         pass_dst(s, pass + 1, hough, tmp));
        st = launched("fht_level_kernel");
    }
    return st;
}
}  // namespace

template <typename In, typename Acc>
int launch_fht_stages(const In *img, int pitch, const Shape &s, Acc *hough, Acc *tmp,
                      cudaStream_t stream) {
    if (s.n == 1) {
        size_t total = (size_t)s.k * 2 * s.W;
        fht_single_row_kernel<In, Acc><<<grid_for(total), 256, 0, stream>>>(img, pitch, s, hough);
        return launched("fht_single_row_kernel");
    }
    fht_level2_kernel<In, Acc><<<s.k * 2 * s.n, 256, 0, stream>>>(img, pitch, s,
                                                                  pass_dst(s, 0, hough, tmp));
    int st = launched("fht_level2_kernel");
    return st ? st : fht_upper_levels<Acc>(s, hough, tmp, stream);
}

template <typename In, typename Acc>
int launch_fht_stages_gauss(const In *img, int pitch, const Shape &s, int r, Acc *hough, Acc *tmp,
                            cudaStream_t stream) {
    dim3 grid((unsigned)(s.k * (s.n / 2)), (unsigned)((s.W + kL2Chunk - 1) / kL2Chunk));
    fht_level2_gauss_kernel<In, Acc><<<grid, 256, 0, stream>>>(
        img, pitch, s, r, binomial_weights(r), pass_dst(s, 0, hough, tmp));
    int st = launched("fht_level2_gauss_kernel");
    return st ? st : fht_upper_levels<Acc>(s, hough, tmp, stream);
}

template int launch_fht_stages_gauss<uint8_t, int32_t>(const uint8_t *, int, const Shape &, int,
                                                       int32_t *, int32_t *, cudaStream_t);
template int launch_fht_stages_gauss<int32_t, int32_t>(const int32_t *, int, const Shape &, int,
                                                       int32_t *, int32_t *, cudaStream_t);
template int launch_fht_stages_gauss<float, float>(const float *, int, const Shape &, int,
                                                   float *, float *, cudaStream_t);
template int launch_fht_stages<uint8_t, int32_t>(const uint8_t *, int, const Shape &, int32_t *,
                                                 int32_t *, cudaStream_t);
template int launch_fht_stages<int32_t, int32_t>(const int32_t *, int, const Shape &, int32_t *,
                                                 int32_t *, cudaStream_t);
template int launch_fht_stages<float, float>(const float *, int, const Shape &, float *, float *,
                                             cudaStream_t);

}  // namespace fhtdp

namespace fhtdp {
namespace {
// Mostly horizontal curves (Sec. 3, Fig. 7) are the mostly vertical curves of
// the transposed image: dst[x][y] = src[y][x], through a 32 x 32 shared tile
// so that both the reads and the writes are row segments.
template <typename T>
__global__ void transpose_kernel(const T *__restrict__ src, int h, int w, int pitch,
                                 T *__restrict__ dst, int dpitch) {
    __shared__ T tile[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int y = y0 + dy, x = x0 + threadIdx.x;
        if (y < h && x < w) tile[dy][threadIdx.x] = src[(size_t)y * pitch + x];
    }
    __syncthreads();
    for (int dx = threadIdx.y; dx < 32; dx += blockDim.y) {
        const int x = x0 + dx, y = y0 + threadIdx.x;
        if (x < w && y < h) dst[(size_t)x * dpitch + y] = tile[threadIdx.x][dx];
    }
}
// The uint8 transpose with 4-byte words: 64 x 64 byte tiles and 16 x 16
// threads; a thread loads one word of each of four tile rows and stores one
// word (four source rows of one column) of each of four output rows.  Needs
// both base addresses and both pitches 4-byte aligned; ragged edges go byte
// by byte.
__global__ void transpose_u8x4_kernel(const uint8_t *__restrict__ src, int h, int w, int pitch,
                                      uint8_t *__restrict__ dst, int dpitch) {
    __shared__ __align__(4) uint8_t tile[64][68];
    const int x0 = blockIdx.x * 64, y0 = blockIdx.y * 64;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int y = y0 + ty + 16 * i, x = x0 + 4 * tx;
        uint32_t v = 0;
        if (y < h) {
            const uint8_t *p = src + (size_t)y * pitch + x;
            if (x + 3 < w) {
                v = *(const uint32_t *)p;
            } else {
                for (int b = 0; b < 4; ++b)
                    if (x + b < w) v |= (uint32_t)p[b] << (8 * b);
            }
        }
        *(uint32_t *)&tile[ty + 16 * i][4 * tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int c = ty + 16 * i, x = x0 + c, y = y0 + 4 * tx;
        if (x >= w || y >= h) continue;
        const uint32_t v = (uint32_t)tile[4 * tx][c] | (uint32_t)tile[4 * tx + 1][c] << 8 |
                           (uint32_t)tile[4 * tx + 2][c] << 16 |
                           (uint32_t)tile[4 * tx + 3][c] << 24;
        uint8_t *q = dst + (size_t)x * dpitch + y;
        if (y + 3 < h) {
            *(uint32_t *)q = v;
        } else {
            for (int b = 0; b < 4 && y + b < h; ++b) q[b] = (uint8_t)(v >> (8 * b));
        }
    }
}
}  // namespace

template <typename T>
int launch_transpose(const T *src, int h, int w, int pitch, T *dst, int dpitch,
                     cudaStream_t stream) {
    if (sizeof(T) == 1 && ((uintptr_t)src & 3) == 0 && ((uintptr_t)dst & 3) == 0 &&
        pitch % 4 == 0 && dpitch % 4 == 0) {
        dim3 grid((unsigned)((w + 63) / 64), (unsigned)((h + 63) / 64));   // h, w <= 2^20
        transpose_u8x4_kernel<<<grid, dim3(16, 16), 0, stream>>>(
            (const uint8_t *)src, h, w, pitch, (uint8_t *)dst, dpitch);
        return launched("transpose_u8x4_kernel");
    }
    dim3 grid((unsigned)((w + 31) / 32), (unsigned)((h + 31) / 32));   // h, w <= 2^20
    transpose_kernel<T><<<grid, dim3(32, 8), 0, stream>>>(src, h, w, pitch, dst, dpitch);
    return launched("transpose_kernel");
}

template int launch_transpose<uint8_t>(const uint8_t *, int, int, int, uint8_t *, int,
                                       cudaStream_t);
template int launch_transpose<int32_t>(const int32_t *, int, int, int, int32_t *, int,
                                       cudaStream_t);
template int launch_transpose<float>(const float *, int, int, int, float *, int, cudaStream_t);

}  // namespace fhtdp
