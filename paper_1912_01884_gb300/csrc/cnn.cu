// The learned shift-window proposal: a 4-layer, 32-channel CNN on a 4x
// downsampled image that predicts, for every band, which of 32 displacement
// bins the best polyline's link falls in; the DP then searches only a window
// around it (pruned DP, with the full DP as fallback).  The paper has no
// counterpart: it is an addition in front of the exact method.
//
// Layout: activations NHWC bf16 ([N][H][W][C], C = 32; the input has C = 1),
// weights bf16 [tap][ci][co] with tap = ky*3 + kx (layer 1: [16][32], taps
// 9..15 zero), FP32 master weights and FP32 accumulation.  The 3x3 dilated
// convolutions ("same" zero padding) run as implicit GEMMs on the tensor
// cores: the 32-channel layers (forward and data gradient) with tcgen05.mma
// (conv_tc.cu), the single-channel first layer and the weight gradient with
// bf16 WMMA 16x16x16 tiles: a CTA takes 64 pixels of one image row and all
// 32 output channels; K = 9 taps x 32 input channels.
#include <mma.h>

#include <cuda_bf16.h>

#include "cnn.cuh"

namespace fhtdp {
namespace {

using namespace nvcuda;

constexpr int kC = 32;        // channels
constexpr int kSeg = 64;      // pixels of a row per CTA
constexpr int kMaxDil = 8;

// ---------------------------------------------------------------------------
// 4x4 mean pool of uint8 images, scaled to [0, 1]: [N][H][W] -> [N][H/4][W/4].
__global__ void downsample4_kernel(const uint8_t *__restrict__ img, long long n_img_stride,
                                   int H, int W, __nv_bfloat16 *__restrict__ out) {
    const int Ho = H / 4, Wo = W / 4;
    const long long total = (long long)gridDim.y * Ho * Wo;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)Ho * Wo;
         i += (long long)gridDim.x * blockDim.x) {
        const int n = blockIdx.y;
        const int yo = (int)(i / Wo), xo = (int)(i % Wo);
        const uint8_t *p = img + n * n_img_stride + (size_t)(4 * yo) * W + 4 * xo;
        unsigned s = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t v = *(const uint32_t *)(p + (size_t)r * W);
            s += (v & 255u) + ((v >> 8) & 255u) + ((v >> 16) & 255u) + (v >> 24);
        }
        out[(size_t)n * Ho * Wo + i] = __float2bfloat16((float)s * (1.0f / (16.0f * 255.0f)));
    }
    (void)total;
}

// ---------------------------------------------------------------------------
// Rows y-dil, y, y+dil of one image, columns [x0 - dil, x0 + kSeg + dil),
// all channels, zero outside the image, into sx[3][kSeg + 2*kMaxDil][kC].
__device__ void stage_rows(const __nv_bfloat16 *X, int cin, int H, int W, int n, int y, int x0,
                           int dil, __nv_bfloat16 *sx) {
    const int width = kSeg + 2 * dil;
    const int per_px = cin;   // 32 or 1
    for (int i = threadIdx.x; i < 3 * width * kC; i += blockDim.x) {
        const int r = i / (width * kC);
        const int rem = i - r * width * kC;
        const int px = rem / kC, c = rem % kC;
        const int yy = y + (r - 1) * dil, xx = x0 - dil + px;
        __nv_bfloat16 v = __float2bfloat16(0.0f);
        if (c < per_px && yy >= 0 && yy < H && xx >= 0 && xx < W)
            v = X[(((size_t)n * H + yy) * W + xx) * per_px + c];
        sx[((size_t)r * (kSeg + 2 * kMaxDil) + px) * kC + c] = v;
    }
}

// One CTA: 64 output pixels x 32 output channels.  8 warps, warp w owns the
// 16x16 output tile (pixels 16*(w/2).., channels 16*(w%2)..).  For cin = 32:
// K = 9 taps x 32 channels; for cin = 1: an im2col tile of the 9 taps
// (padded to 16) and one K step.  out = act(sum + bias), bf16.
template <bool kRelu>
__global__ void __launch_bounds__(256) conv3x3_kernel(const __nv_bfloat16 *__restrict__ X,
                                                      int cin, int H, int W, int dil,
                                                      const __nv_bfloat16 *__restrict__ Wt,
                                                      const float *__restrict__ bias,
                                                      __nv_bfloat16 *__restrict__ Y) {
    __shared__ __align__(128) __nv_bfloat16 sx[3 * (kSeg + 2 * kMaxDil) * kC];
    __shared__ __align__(128) __nv_bfloat16 sw[9 * kC * kC];
    __shared__ __align__(128) float so[kSeg * kC];
    const int segs = W / kSeg;
    const int n = blockIdx.x / (H * segs);
    const int rem = blockIdx.x % (H * segs);
    const int y = rem / segs, x0 = (rem % segs) * kSeg;
    const int warp = threadIdx.x >> 5;
    const int pb = warp >> 1, cb = warp & 1;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
    wmma::fill_fragment(acc, 0.0f);
    if (cin == kC) {
        for (int i = threadIdx.x; i < 9 * kC * kC; i += blockDim.x) sw[i] = Wt[i];
        stage_rows(X, cin, H, W, n, y, x0, dil, sx);
        __syncthreads();
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
            for (int c0 = 0; c0 < kC; c0 += 16) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> a;
                wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> b;
                const __nv_bfloat16 *ap =
                    sx + ((size_t)ky * (kSeg + 2 * kMaxDil) + 16 * pb + kx * dil) * kC + c0;
                wmma::load_matrix_sync(a, ap, kC);
                wmma::load_matrix_sync(b, sw + ((size_t)tap * kC + c0) * kC + 16 * cb, kC);
                wmma::mma_sync(acc, a, b, acc);
            }
        }
    } else {
        // im2col of the single input channel: sx as [kSeg][16] (k = tap).
        __nv_bfloat16 *col = sx;
        for (int i = threadIdx.x; i < 16 * kC; i += blockDim.x) sw[i] = Wt[i];
        for (int i = threadIdx.x; i < kSeg * 16; i += blockDim.x) {
            const int p = i / 16, k = i % 16;
            __nv_bfloat16 v = __float2bfloat16(0.0f);
            if (k < 9) {
                const int yy = y + (k / 3 - 1) * dil, xx = x0 + p + (k % 3 - 1) * dil;
                if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = X[((size_t)n * H + yy) * W + xx];
            }
            col[i] = v;
        }
        __syncthreads();
        wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> a;
        wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> b;
        wmma::load_matrix_sync(a, col + 16 * pb * 16, 16);
        wmma::load_matrix_sync(b, sw + 16 * cb, kC);
        wmma::mma_sync(acc, a, b, acc);
    }
    wmma::store_matrix_sync(so + (16 * pb) * kC + 16 * cb, acc, kC, wmma::mem_row_major);
    __syncthreads();
    for (int i = threadIdx.x; i < kSeg * kC; i += blockDim.x) {
        const int p = i / kC, c = i % kC;
        float v = so[i] + (bias ? bias[c] : 0.0f);
        if (kRelu) v = v > 0.0f ? v : 0.0f;
        Y[(((size_t)n * H + y) * W + x0 + p) * kC + c] = __float2bfloat16(v);
    }
}

// ---------------------------------------------------------------------------
// dZ = dY * (Y > 0) in place (the ReLU of a layer, from its output).
__global__ void relu_backward_kernel(const __nv_bfloat16 *__restrict__ Y,
                                     __nv_bfloat16 *__restrict__ dY, long long count) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(Y[i]) > 0.0f)) dY[i] = __float2bfloat16(0.0f);
}

// Weights of the data gradient: W'[tap'][co][ci] = W[8 - tap'][ci][co].
__global__ void flip_transpose_kernel(const __nv_bfloat16 *__restrict__ Wt,
                                      __nv_bfloat16 *__restrict__ Wf) {
    for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < 9 * kC * kC;
         i += blockDim.x * gridDim.x) {
        const int tap = i / (kC * kC), r = i % (kC * kC);
        const int co = r / kC, ci = r % kC;
        Wf[i] = Wt[((size_t)(8 - tap) * kC + ci) * kC + co];
    }
}

// ---------------------------------------------------------------------------
// Weight and bias gradients: dW[tap][ci][co] += sum_p X(p + off(tap))[ci] *
// dZ(p)[co], db[co] += sum_p dZ(p)[co].  Persistent CTAs loop over row
// segments and keep their partial sums in tensor-core accumulators; one
// atomic flush per CTA.  8 warps share the 18 (tap, ci block) x 2 (co block)
// output tiles of a 32-channel input (cin = 1: the 1 x 2 tiles of the
// im2col form).
__global__ void __launch_bounds__(256) conv3x3_wgrad_kernel(const __nv_bfloat16 *__restrict__ X,
                                                            int cin, int N, int H, int W,
                                                            int dil,
                                                            const __nv_bfloat16 *__restrict__ dZ,
                                                            float *__restrict__ dW,
                                                            float *__restrict__ db) {
    __shared__ __align__(128) __nv_bfloat16 sx[3 * (kSeg + 2 * kMaxDil) * kC];
    __shared__ __align__(128) __nv_bfloat16 sz[kSeg * kC];
    __shared__ __align__(128) float sacc[16 * 16 * 8];
    const int warp = threadIdx.x >> 5;
    const int tiles = cin == kC ? 36 : 2;
    constexpr int kMaxTiles = 5;   // ceil(36 / 8)
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[kMaxTiles];
#pragma unroll
    for (int t = 0; t < kMaxTiles; ++t) wmma::fill_fragment(acc[t], 0.0f);
    float bsum = 0.0f;   // thread c < 32: bias gradient of channel c
    const int segs = W / kSeg;
    const long long units = (long long)N * H * segs;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const int n = (int)(u / (H * segs));
        const int rem = (int)(u % (H * segs));
        const int y = rem / segs, x0 = (rem % segs) * kSeg;
        __syncthreads();
        for (int i = threadIdx.x; i < kSeg * kC; i += blockDim.x)
            sz[i] = dZ[(((size_t)n * H + y) * W + x0) * kC + i];
        if (cin == kC) {
            stage_rows(X, cin, H, W, n, y, x0, dil, sx);
        } else {
            for (int i = threadIdx.x; i < kSeg * 16; i += blockDim.x) {
                const int p = i / 16, k = i % 16;
                __nv_bfloat16 v = __float2bfloat16(0.0f);
                if (k < 9) {
                    const int yy = y + (k / 3 - 1) * dil, xx = x0 + p + (k % 3 - 1) * dil;
                    if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                        v = X[((size_t)n * H + yy) * W + xx];
                }
                sx[i] = v;
            }
        }
        __syncthreads();
        if (threadIdx.x < kC)
            for (int p = 0; p < kSeg; ++p) bsum += __bfloat162float(sz[p * kC + threadIdx.x]);
#pragma unroll
        for (int t = 0; t < kMaxTiles; ++t) {
            const int tile = warp + 8 * t;
            if (tile >= tiles) break;
            const int kb = tile >> 1, cb = tile & 1;   // kb: (tap, ci block) or 0
            for (int p0 = 0; p0 < kSeg; p0 += 16) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::col_major> a;
                wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> b;
                if (cin == kC) {
                    const int tap = kb >> 1, c0 = 16 * (kb & 1);
                    const int ky = tap / 3, kx = tap % 3;
                    // A = X^T: rows = input channels, columns = pixels.
                    wmma::load_matrix_sync(
                        a, sx + ((size_t)ky * (kSeg + 2 * kMaxDil) + p0 + kx * dil) * kC + c0, kC);
                } else {
                    wmma::load_matrix_sync(a, sx + p0 * 16, 16);
                }
                wmma::load_matrix_sync(b, sz + p0 * kC + 16 * cb, kC);
                wmma::mma_sync(acc[t], a, b, acc[t]);
            }
        }
    }
    // Flush: dW rows k = tap * 32 + ci (cin = 32) or k = tap (cin = 1).
    float *st = sacc + warp * 256;
#pragma unroll
    for (int t = 0; t < kMaxTiles; ++t) {
        const int tile = warp + 8 * t;
        if (tile >= tiles) break;
        const int kb = tile >> 1, cb = tile & 1;
        wmma::store_matrix_sync(st, acc[t], 16, wmma::mem_row_major);
        __syncwarp();
        for (int i = threadIdx.x & 31; i < 256; i += 32) {
            const int r = i / 16, c = i % 16;
            const int k = 16 * kb + r;
            atomicAdd(&dW[(size_t)k * kC + 16 * cb + c], st[i]);
        }
        __syncwarp();
    }
    if (threadIdx.x < kC && db) atomicAdd(&db[threadIdx.x], bsum);
}

// ---------------------------------------------------------------------------
// Band head: for image n and band b (rows [b*rpb, (b+1)*rpb) of the low-res
// logits), pooled[c] = log sum_{rows, cols} exp(logit[c]) (a smooth maximum
// over the band), the softmax cross-entropy of the 32 pooled logits against
// the label bin, its gradient dlogit = (softmax - onehot)[c] *
// exp(logit - pooled[c]) * scale, and the predicted bin.
__global__ void __launch_bounds__(256) band_head_kernel(const __nv_bfloat16 *__restrict__ L,
                                                        int H, int W, int bands,
                                                        const int32_t *__restrict__ labels,
                                                        float scale,
                                                        __nv_bfloat16 *__restrict__ dL,
                                                        float *__restrict__ loss,
                                                        int32_t *__restrict__ pred,
                                                        float *__restrict__ conf) {
    __shared__ float smax[8][kC], ssum[8][kC], pooled[kC], dpool[kC];
    const int n = blockIdx.x / bands, b = blockIdx.x % bands;
    const int rpb = H / bands;
    const int c = threadIdx.x & 31, part = threadIdx.x >> 5;
    const int positions = rpb * W;
    const __nv_bfloat16 *base = L + ((size_t)n * H + (size_t)b * rpb) * W * kC;
    float m = -INFINITY, s = 0.0f;
    for (int pidx = part; pidx < positions; pidx += 8) {
        const float v = __bfloat162float(base[(size_t)pidx * kC + c]);
        if (v > m) {
            s = s * __expf(m - v) + 1.0f;
            m = v;
        } else {
            s += __expf(v - m);
        }
    }
    smax[part][c] = m;
    ssum[part][c] = s;
    __syncthreads();
    if (threadIdx.x < kC) {
        float M = -INFINITY;
        for (int p = 0; p < 8; ++p) M = fmaxf(M, smax[p][c]);
        float S = 0.0f;
        for (int p = 0; p < 8; ++p) S += ssum[p][c] * __expf(smax[p][c] - M);
        pooled[c] = M + __logf(S);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float M = -INFINITY;
        int arg = 0;
        for (int k = 0; k < kC; ++k)
            if (pooled[k] > M) {
                M = pooled[k];
                arg = k;
            }
        float S = 0.0f;
        for (int k = 0; k < kC; ++k) S += __expf(pooled[k] - M);
        const float lse = M + __logf(S);
        const int lab = labels ? labels[n * bands + b] : -1;
        for (int k = 0; k < kC; ++k) dpool[k] = __expf(pooled[k] - lse) - (k == lab ? 1.0f : 0.0f);
        if (loss && lab >= 0) atomicAdd(loss, (lse - pooled[lab]) * scale);
        if (pred) pred[n * bands + b] = arg;
        if (conf) conf[n * bands + b] = __expf(M - lse);   // softmax probability of the argmax
    }
    __syncthreads();
    if (!dL) return;
    __nv_bfloat16 *dbase = dL + ((size_t)n * H + (size_t)b * rpb) * W * kC;
    const float pc = pooled[c], g = dpool[c] * scale;
    for (int pidx = part; pidx < positions; pidx += 8) {
        const float v = __bfloat162float(base[(size_t)pidx * kC + c]);
        dbase[(size_t)pidx * kC + c] = __float2bfloat16(g * __expf(v - pc));
    }
}

// ---------------------------------------------------------------------------
// Adam on FP32 master parameters; refreshes the bf16 copy used by the
// forward pass (when `wb` is given).
__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, int count, float lr, float b1, float b2,
                            float eps, float c1, float c2, __nv_bfloat16 *__restrict__ wb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = pi;
        if (wb) wb[i] = __float2bfloat16(pi);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst,
                               int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16(src[i]);
}

// Displacement windows from the predicted bins: bin c covers d + 64 in
// [4c, 4c + 3]; the window is those 4 values with `margin` more on each side,
// clipped to [-(n-1), n-1].
__global__ void bin_windows_kernel(const int32_t *__restrict__ pred, int count, int n, int margin,
                                   int32_t *__restrict__ win) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const int lo = 4 * pred[i] - 64 - margin, hi = 4 * pred[i] - 61 + margin;
        win[2 * i] = lo < -(n - 1) ? -(n - 1) : lo;
        win[2 * i + 1] = hi > n - 1 ? n - 1 : hi;
    }
}

// He-normal initial weights (standard deviation sqrt(2 / fan_in)) from a
// counter-based SplitMix64 stream (Steele, Lea, Flood, OOPSLA 2014) and the
// Box-Muller transform; zero where `zero_from` <= row (padding taps).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void he_init_kernel(float *__restrict__ w, int rows, int cols, int zero_from, float std,
                               unsigned long long seed) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols;
         i += gridDim.x * blockDim.x) {
        const unsigned long long r1 = splitmix64(seed ^ (2ull * (unsigned long long)i));
        const unsigned long long r2 = splitmix64(seed ^ (2ull * (unsigned long long)i + 1ull));
        const float u1 = ((float)(r1 >> 40) + 0.5f) * (1.0f / 16777216.0f);
        const float u2 = (float)(r2 >> 40) * (1.0f / 16777216.0f);
        const float z = sqrtf(-2.0f * logf(u1)) * cosf(6.283185307179586f * u2);
        w[i] = (i / cols) >= zero_from ? 0.0f : std * z;
    }
}

int grid_1d(long long count, int block) {
    long long g = (count + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

bool cnn_shape_ok(int H, int W, int dil) {
    return H >= 1 && W >= kSeg && W % kSeg == 0 && dil >= 1 && dil <= kMaxDil;
}

int cnn_downsample4(const uint8_t *img, int N, int H, int W, void *out, cudaStream_t stream) {
    dim3 grid(grid_1d((long long)(H / 4) * (W / 4), 256), N);
    downsample4_kernel<<<grid, 256, 0, stream>>>(img, (long long)H * W, H, W,
                                                 (__nv_bfloat16 *)out);
    return launched("downsample4_kernel");
}

int cnn_conv3x3(const void *X, int cin, int N, int H, int W, int dil, const void *Wt,
                const float *bias, int relu, void *Y, cudaStream_t stream) {
    // 32 input channels: the tcgen05 kernel; the single-channel first layer
    // (1/32 of the work) keeps the WMMA one
    if (cin == kC) return cnn_conv3x3_tc(X, N, H, W, dil, Wt, bias, relu, Y, stream);
    const long long blocks = (long long)N * H * (W / kSeg);
    if (relu)
        conv3x3_kernel<true><<<(unsigned)blocks, 256, 0, stream>>>(
            (const __nv_bfloat16 *)X, cin, H, W, dil, (const __nv_bfloat16 *)Wt, bias,
            (__nv_bfloat16 *)Y);
    else
        conv3x3_kernel<false><<<(unsigned)blocks, 256, 0, stream>>>(
            (const __nv_bfloat16 *)X, cin, H, W, dil, (const __nv_bfloat16 *)Wt, bias,
            (__nv_bfloat16 *)Y);
    return launched("conv3x3_kernel");
}

int cnn_relu_backward(const void *Y, void *dY, long long count, cudaStream_t stream) {
    relu_backward_kernel<<<grid_1d(count, 256), 256, 0, stream>>>(
        (const __nv_bfloat16 *)Y, (__nv_bfloat16 *)dY, count);
    return launched("relu_backward_kernel");
}

int cnn_flip_transpose(const void *Wt, void *Wf, cudaStream_t stream) {
    flip_transpose_kernel<<<36, 256, 0, stream>>>((const __nv_bfloat16 *)Wt, (__nv_bfloat16 *)Wf);
    return launched("flip_transpose_kernel");
}

int cnn_wgrad(const void *X, int cin, int N, int H, int W, int dil, const void *dZ, float *dW,
              float *db, cudaStream_t stream) {
    if (cin == kC) return cnn_wgrad_tc(X, N, H, W, dil, dZ, dW, db, stream);
    conv3x3_wgrad_kernel<<<2 * 152, 256, 0, stream>>>((const __nv_bfloat16 *)X, cin, N, H, W, dil,
                                                      (const __nv_bfloat16 *)dZ, dW, db);
    return launched("conv3x3_wgrad_kernel");
}

int cnn_band_head(const void *L, int N, int H, int W, int bands, const int32_t *labels,
                  float scale, void *dL, float *loss, int32_t *pred, cudaStream_t stream,
                  float *conf) {
    band_head_kernel<<<N * bands, 256, 0, stream>>>((const __nv_bfloat16 *)L, H, W, bands, labels,
                                                     scale, (__nv_bfloat16 *)dL, loss, pred, conf);
    return launched("band_head_kernel");
}

int cnn_adam(float *p, float *m, float *v, const float *g, int count, float lr, float b1,
             float b2, float eps, int t, void *wb, cudaStream_t stream) {
    const float c1 = 1.0f / (1.0f - powf(b1, (float)t)), c2 = 1.0f / (1.0f - powf(b2, (float)t));
    adam_kernel<<<grid_1d(count, 256), 256, 0, stream>>>(p, m, v, g, count, lr, b1, b2, eps, c1,
                                                        c2, (__nv_bfloat16 *)wb);
    return launched("adam_kernel");
}

int cnn_bin_windows(const int32_t *pred, int count, int n, int margin, int32_t *win,
                    cudaStream_t stream) {
    bin_windows_kernel<<<grid_1d(count, 256), 256, 0, stream>>>(pred, count, n, margin, win);
    return launched("bin_windows_kernel");
}

int cnn_he_init(float *w, int rows, int cols, int zero_from, float std, unsigned long long seed,
                cudaStream_t stream) {
    he_init_kernel<<<grid_1d((long long)rows * cols, 256), 256, 0, stream>>>(w, rows, cols,
                                                                           zero_from, std, seed);
    return launched("he_init_kernel");
}

int cnn_to_bf16(const float *src, void *dst, int count, cudaStream_t stream) {
    to_bf16_kernel<<<grid_1d(count, 256), 256, 0, stream>>>(src, (__nv_bfloat16 *)dst, count);
    return launched("to_bf16_kernel");
}

}  // namespace fhtdp
