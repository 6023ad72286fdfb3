// 3x3 dilated convolutions of the learned window proposal with 32 input and
// 32 output channels on the fifth-generation tensor cores (tcgen05.mma,
// accumulators in tensor memory).  The paper has no counterpart: the network
// is an addition in front of the exact method.
//
// A tile is 128 output pixels of one image row for all 32 output channels:
// an implicit GEMM D[p][co] = sum over taps t and input channels ci of
// X(p + off(t))[ci] * W[t][ci][co], M = 128, N = 32, K = 9 x 32, as 18 MMAs of
// K = 16 (bf16 operands, FP32 accumulation).  Persistent CTAs (4 warps, three
// per SM) load the weights once and pipeline their tiles (see
// conv3x3_tc_persist_kernel).
//
// Shared memory holds operands in the no-swizzle K-major layout of the MMA:
// "core matrices" of 8 rows x 16 bytes (8 bf16 along K) stored as 128
// contiguous bytes.
//  - A: the three input rows y - dil, y, y + dil, pixels [x0 - 8, x0 + 136)
//    (zero outside the image), as [row][channel chunk][pixel][8 channels]:
//    rows of a core matrix are consecutive pixels (16 bytes apart), the next
//    8 pixels 128 bytes on, the next channel chunk kAChunk bytes on.  The
//    operand of tap (ky, kx) is the same buffer from pixel 8 + (kx - 1) * dil:
//    every tap reads the staged rows in place.
//  - B: the weights as [tap][channel chunk][co][8 ci] (512 bytes per chunk).
// D (128 lanes x 32 FP32 columns of tensor memory) is read back by the four
// warps, one lane quarter each (tcgen05.ld 32x32b), then bias, ReLU and bf16.
#include <cuda_bf16.h>

#include <algorithm>

#include "cnn.cuh"

namespace fhtdp {
namespace {

constexpr int kTcC = 32;                 // channels
constexpr int kTcM = 128;                // output pixels of a CTA
constexpr int kTcHalo = 8;               // largest dilation
constexpr int kTcPix = kTcM + 2 * kTcHalo;             // staged pixels of a row
constexpr int kAChunk = kTcPix * 16;                    // bytes of one channel chunk
constexpr int kARow = 4 * kAChunk;                      // bytes of one staged row
constexpr int kABytes = 3 * kARow;                      // 27,648
constexpr int kBBytes = 9 * 4 * kTcC * 16;              // 18,432
constexpr int kTcThreads = 128;
constexpr unsigned kTmemCols = 32;

// Device status of the tensor-core convolutions: FHTDP_ETIMEOUT once a
// bounded wait for the MMAs gave up (read with fhtdp_cnn_status).
__device__ int g_conv_tc_status;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading and
// stride byte offsets of the core matrices, each in 16-byte units; bit 46 is
// the descriptor version.  Without swizzling the leading offset is the step
// between core matrices along K and the stride offset the step along M / N,
// for K-major and MN-major operands alike.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3ffffu) >> 4) | ((uint64_t)((lbo & 0x3ffffu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3ffffu) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), bf16
// A and B (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at
// bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcC >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
// Bounded parity wait: false when `limit` cycles passed first.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    // src-size 0 fills the 16 bytes with zeros
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

// The forward as a persistent kernel: a CTA loads the weights once and takes
// the tiles (image, row, 128-pixel segment) u = blockIdx.x, blockIdx.x +
// gridDim.x, ...  Two stage buffers and two accumulators (64 columns of tensor
// memory) overlap the MMAs of tile i with the loads of tile i+1 and the
// epilogue of tile i-1:
//   wait for tile i's rows; MMAs of tile i into accumulator i % 2;
//   wait for tile i-1's MMAs, its epilogue from accumulator (i-1) % 2;
//   the rows of tile i+1 into the stage tile i-1 used.
__device__ __forceinline__ void tc_tile_coords(long long u, int H, int segs, int *n, int *y,
                                               int *x0) {
    *n = (int)(u / ((long long)H * segs));
    const int rem = (int)(u % ((long long)H * segs));
    *y = rem / segs;
    *x0 = (rem % segs) * kTcM;
}

// All threads: the three rows of tile (n, y, x0) into stage As (cp.async,
// zero outside the image), one commit group.
__device__ __forceinline__ void tc_stage_rows(const __nv_bfloat16 *X, int H, int W, int dil, int n,
                                              int y, int x0, unsigned char *As) {
    for (int i = threadIdx.x; i < 3 * 4 * kTcPix; i += kTcThreads) {
        const int c = i & 3, q = (i >> 2) % kTcPix, r = (i >> 2) / kTcPix;
        const int yy = y + (r - 1) * dil, xx = x0 - kTcHalo + q;
        const bool ok = yy >= 0 && yy < H && xx >= 0 && xx < W;
        const __nv_bfloat16 *src =
            ok ? X + ((((size_t)n * H + yy) * W + xx) * kTcC + 8 * c) : X;
        cp_async16(smem_u32(As + r * kARow + c * kAChunk + q * 16), src, ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Thread 0: the 18 MMAs of one tile from stage As and the weights Bs into
// accumulator `acc_tmem`, completion on `bar`.
__device__ __forceinline__ void tc_issue(const unsigned char *As, const unsigned char *Bs,
                                         int dil, uint32_t acc_tmem, uint64_t *bar) {
    const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
    for (int t = 0; t < 9; ++t) {
        const int ky = t / 3, kx = t % 3;
        const uint32_t abase = a0 + ky * kARow + (kTcHalo + (kx - 1) * dil) * 16;
        for (int j = 0; j < 2; ++j) {
            const uint64_t ad = sdesc(abase + 2 * j * kAChunk, kAChunk, 128);
            const uint64_t bd = sdesc(b0 + (t * 4 + 2 * j) * 512, 512, 128);
            const uint32_t acc = (t | j) != 0;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_tmem),
                "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                : "memory");
        }
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// All threads: the epilogue of a tile from accumulator `acc_tmem` (warp w
// reads lanes 32w..32w+31, i.e. pixels x0 + 32w + lane): bias, ReLU, bf16.
template <bool kRelu>
__device__ __forceinline__ void tc_epilogue(uint32_t acc_tmem, const float *bias,
                                            __nv_bfloat16 *Y, int H, int W, int n, int y,
                                            int x0) {
    const int warp = threadIdx.x >> 5;
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(acc_tmem + ((uint32_t)(32 * warp) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int x = x0 + threadIdx.x;
    if (x >= W) return;
    uint32_t packed[16];
#pragma unroll
    for (int c = 0; c < kTcC; c += 2) {
        float v0 = __uint_as_float(r[c]) + (bias ? __ldg(bias + c) : 0.0f);
        float v1 = __uint_as_float(r[c + 1]) + (bias ? __ldg(bias + c + 1) : 0.0f);
        if (kRelu) {
            v0 = v0 > 0.0f ? v0 : 0.0f;
            v1 = v1 > 0.0f ? v1 : 0.0f;
        }
        const __nv_bfloat162 hv = __floats2bfloat162_rn(v0, v1);
        packed[c / 2] = *(const uint32_t *)&hv;
    }
    uint4 *dst = (uint4 *)(Y + (((size_t)n * H + y) * W + x) * kTcC);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
}

template <bool kRelu>
__global__ void __launch_bounds__(kTcThreads) conv3x3_tc_persist_kernel(
    const __nv_bfloat16 *__restrict__ X, int N, int H, int W, int dil,
    const __nv_bfloat16 *__restrict__ Wt, const float *__restrict__ bias,
    __nv_bfloat16 *__restrict__ Y, long long wait_cycles) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Bs = smem;                       // weights
    unsigned char *As[2] = {smem + kBBytes, smem + kBBytes + kABytes};   // stages
    __shared__ __align__(8) uint64_t s_done[2];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int segs = (W + kTcM - 1) / kTcM;
    const long long units = (long long)N * H * segs;
    if (tid == 0) {
        mbar_init(&s_done[0], 1);
        mbar_init(&s_done[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(2 * kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < 9 * kTcC * kTcC; i += kTcThreads) {
        const int co = i & 31, ci = (i >> 5) & 31, t = i >> 10;
        ((__nv_bfloat16 *)Bs)[((t * 4 + (ci >> 3)) * kTcC + co) * 8 + (ci & 7)] = Wt[i];
    }
    int n, y, x0;
    if (blockIdx.x < units) {
        tc_tile_coords(blockIdx.x, H, segs, &n, &y, &x0);
        tc_stage_rows(X, H, W, dil, n, y, x0, As[0]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    uint32_t ph[2] = {0u, 0u};
    long long prev = -1;
    int b = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < units; u += gridDim.x, b ^= 1) {
        // tile u's rows (and, the first time, the weights) -> the tensor core
        asm volatile("cp.async.wait_all;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) tc_issue(As[b], Bs, dil, tmem + kTmemCols * b, &s_done[b]);
        __syncwarp();
        if (prev >= 0) {   // tile prev: its MMAs, then its epilogue
            const bool w = mbar_wait(&s_done[b ^ 1], ph[b ^ 1], wait_cycles);
            if (!w) {
                if (lane == 0) atomicExch(&g_conv_tc_status, FHTDP_ETIMEOUT);
                mbar_wait(&s_done[b ^ 1], ph[b ^ 1], 4 * wait_cycles);
            }
            ph[b ^ 1] ^= 1u;
            ok = __syncthreads_and(w) != 0;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_tile_coords(prev, H, segs, &n, &y, &x0);
            tc_epilogue<kRelu>(tmem + kTmemCols * (b ^ 1), bias, Y, H, W, n, y, x0);
        }
        // the stage tile prev read is free: the rows of the next tile
        const long long next = u + gridDim.x;
        if (next < units) {
            tc_tile_coords(next, H, segs, &n, &y, &x0);
            tc_stage_rows(X, H, W, dil, n, y, x0, As[b ^ 1]);
        }
        prev = u;
    }
    if (ok && prev >= 0) {   // the last tile took accumulator b ^ 1
        const bool w = mbar_wait(&s_done[b ^ 1], ph[b ^ 1], wait_cycles);
        if (!w) {
            if (lane == 0) atomicExch(&g_conv_tc_status, FHTDP_ETIMEOUT);
            mbar_wait(&s_done[b ^ 1], ph[b ^ 1], 4 * wait_cycles);
        }
        if (__syncthreads_and(w)) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_tile_coords(prev, H, segs, &n, &y, &x0);
            tc_epilogue<kRelu>(tmem + kTmemCols * (b ^ 1), bias, Y, H, W, n, y, x0);
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * kTmemCols)
                     : "memory");
}

// Weight and bias gradients of a 32-channel layer: dW[t][ci][co] += sum over
// pixels p of X(p + off(t))[ci] * dZ(p)[co], db[co] += sum of dZ(p)[co].  As
// GEMMs with the pixels as K, one per column tap kx: M = 128 rows (ky, ci) for
// ky = 0..3, N = 32 (co).  The A operand is the forward kernel's stage of the
// three input rows y - dil, y, y + dil ([row][channel chunk][pixel][8 ci],
// pixels [x0 - 8, x0 + 136)) read in place from pixel 8 + (kx - 1) dil, so a
// segment is copied once for all nine taps; a fourth staged "row" holds a
// chunk of ones, so accumulator rows 96..103 of every tap group are db, and
// rows 104..127 (its other chunks, never written) are never read.  Both
// operands are MN-major (channels contiguous, as stored): core matrices of 8
// channels (16 bytes) x 8 pixels; for A the next 8 rows of M are kAChunk
// bytes on (row ky of the stage is four chunks on) and the next 8 pixels of K
// 128 bytes on; B is dZ as [chunk][pixel][8 co] (kWgChunk, 128).
// Persistent CTAs (4 warps, two per SM) walk 128-pixel row segments through
// two stages: segment i + 1's copies are in flight while segment i's land and
// segment i - 1's MMAs run; the three accumulators (96 columns of tensor
// memory) stay put, and at the end warp ky adds its row's 32 values of each
// tap group to dW (warp 3: db).
constexpr int kWgP = kTcM;                      // pixels of a segment (K per stage)
constexpr int kWgChunk = kWgP * 16;             // bytes of a chunk of dZ
constexpr int kWgABytes = 4 * kARow;            // 36,864: three rows and the ones
constexpr int kWgBBytes = 4 * kWgChunk;         // 8,192
constexpr int kWgStage = kWgABytes + kWgBBytes; // 45,056
constexpr int kWgThreads = kTcThreads;
constexpr unsigned kWgCols = 128;               // three 32-column accumulators
constexpr uint32_t kIdescMN = kIdesc | (1u << 15) | (1u << 16);   // A and B MN-major

// cp.async of segment u (image, row, 128 pixels) into one stage: the three
// rows of X (zero outside the image) and dZ (zero past the row's end).
__device__ __forceinline__ void wg_stage(const __nv_bfloat16 *X, const __nv_bfloat16 *dZ, int H,
                                         int W, int dil, int segs, long long u,
                                         unsigned char *st) {
    int n, y, x0;
    tc_tile_coords(u, H, segs, &n, &y, &x0);
    for (int i = threadIdx.x; i < 3 * 4 * kTcPix; i += kWgThreads) {
        const int c = i & 3, q = (i >> 2) % kTcPix, r = (i >> 2) / kTcPix;
        const int yy = y + (r - 1) * dil, xx = x0 - kTcHalo + q;
        const bool v = yy >= 0 && yy < H && xx >= 0 && xx < W;
        const __nv_bfloat16 *src = v ? X + ((((size_t)n * H + yy) * W + xx) * kTcC + 8 * c) : X;
        cp_async16(smem_u32(st + r * kARow + c * kAChunk + q * 16), src, v);
    }
    for (int i = threadIdx.x; i < 4 * kWgP; i += kWgThreads) {
        const int c = i & 3, p = i >> 2;
        const bool v = x0 + p < W;
        const __nv_bfloat16 *src = v ? dZ + ((((size_t)n * H + y) * W + x0 + p) * kTcC + 8 * c) : dZ;
        cp_async16(smem_u32(st + kWgABytes + c * kWgChunk + p * 16), src, v);
    }
}

__global__ void __launch_bounds__(kWgThreads) conv3x3_wgrad_tc_kernel(
    const __nv_bfloat16 *__restrict__ X, int N, int H, int W, int dil,
    const __nv_bfloat16 *__restrict__ dZ, float *__restrict__ dW, float *__restrict__ db,
    long long wait_cycles) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *St[2] = {smem, smem + kWgStage};
    __shared__ __align__(8) uint64_t s_done[2];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&s_done[0], 1);
        mbar_init(&s_done[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kWgCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the ones chunk (row 3, chunk 0) of both stages, bf16 1.0 = 0x3f80; the
    // stage copies never write it
    for (int i = tid; i < 2 * kTcPix; i += kWgThreads)
        *(uint4 *)(St[i / kTcPix] + 3 * kARow + (i % kTcPix) * 16) =
            make_uint4(0x3f803f80u, 0x3f803f80u, 0x3f803f80u, 0x3f803f80u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const int segs = (W + kWgP - 1) / kWgP;
    const long long units = (long long)N * H * segs;
    uint32_t ph[2] = {0u, 0u};
    bool pend[2] = {false, false};
    bool first = true, ok = true;
    long long u = blockIdx.x;
    int b = 0;
    if (u < units) wg_stage(X, dZ, H, W, dil, segs, u, St[0]);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (; u < units; u += gridDim.x, b ^= 1) {
        const long long nu = u + gridDim.x;
        if (nu < units) {
            // stage b ^ 1 is rewritten: wait for the MMAs that read it
            if (pend[b ^ 1]) {
                const bool w = mbar_wait(&s_done[b ^ 1], ph[b ^ 1], wait_cycles);
                if (!w) {
                    if (lane == 0) atomicExch(&g_conv_tc_status, FHTDP_ETIMEOUT);
                    mbar_wait(&s_done[b ^ 1], ph[b ^ 1], 4 * wait_cycles);
                }
                ph[b ^ 1] ^= 1u;
                pend[b ^ 1] = false;
                ok = __syncthreads_and(w) != 0;
                if (!ok) break;
            }
            wg_stage(X, dZ, H, W, dil, segs, nu, St[b ^ 1]);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");   // stage b has landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t a0 = smem_u32(St[b]), b0 = a0 + kWgABytes;
            for (int g = 0; g < 3; ++g)   // column tap kx = g
                for (int j = 0; j < kWgP / 16; ++j) {
                    // MN-major, no swizzle: the leading offset steps along K
                    // (8 pixels), the stride offset along M / N (8 channels)
                    const uint32_t abase = a0 + (kTcHalo + (g - 1) * dil) * 16;
                    const uint64_t ad = sdesc(abase + j * 256, 128, kAChunk);
                    const uint64_t bd = sdesc(b0 + j * 256, 128, kWgChunk);
                    const uint32_t acc = first && j == 0 ? 0u : 1u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                            tmem + 32u * g),
                        "l"(ad), "l"(bd), "r"(kIdescMN), "r"(acc)
                        : "memory");
                }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&s_done[b]))
                : "memory");
        }
        __syncwarp();
        pend[b] = true;
        first = false;
    }
    // the MMAs complete in order: wait for the pending ones (both stages)
    for (int s = 0; s < 2 && ok; ++s)
        if (pend[s]) {
            const bool w = mbar_wait(&s_done[s], ph[s], wait_cycles);
            if (!w) {
                if (lane == 0) atomicExch(&g_conv_tc_status, FHTDP_ETIMEOUT);
                mbar_wait(&s_done[s], ph[s], 4 * wait_cycles);
            }
            ok = __syncthreads_and(w) != 0;
        }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!first && ok) {
        // row 32 warp + lane of group g is tap 3 warp + g (ky = warp, kx = g),
        // input channel lane; warp 3, lanes 0..7 hold db
        for (int g = 0; g < 3; ++g) {
            const int t = 3 * warp + g;
            uint32_t r[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
                "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, "
                "%26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                  "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                  "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                  "=r"(r[30]), "=r"(r[31])
                : "r"(tmem + ((uint32_t)(32 * warp) << 16) + 32u * g));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (warp < 3) {
                float *dst = dW + ((size_t)t * kTcC + lane) * kTcC;
#pragma unroll
                for (int co = 0; co < kTcC; ++co) atomicAdd(dst + co, __uint_as_float(r[co]));
            } else if (g == 0 && lane == 0 && db) {
#pragma unroll
                for (int co = 0; co < kTcC; ++co) atomicAdd(db + co, __uint_as_float(r[co]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kWgCols)
                     : "memory");
}

}  // namespace

int cnn_wgrad_tc(const void *X, int N, int H, int W, int dil, const void *dZ, float *dW,
                 float *db, cudaStream_t stream) {
    if (dil < 1 || dil > kTcHalo || W < 1 || H < 1 || N < 1)
        return set_error(FHTDP_EINVAL, "conv3x3 wgrad: dilation 1..8 and a non-empty image");
    const size_t smem = 2 * (size_t)kWgStage;
    // set on every call: the attribute belongs to the current device
    int st = cuda_status(cudaFuncSetAttribute(conv3x3_wgrad_tc_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem),
                         "cudaFuncSetAttribute");
    if (st) return st;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long units = (long long)N * H * ((W + kWgP - 1) / kWgP);
    const long long grid = std::min<long long>(units, 2LL * (sms > 0 ? sms : 152));
    conv3x3_wgrad_tc_kernel<<<(unsigned)grid, kWgThreads, smem, stream>>>(
        (const __nv_bfloat16 *)X, N, H, W, dil, (const __nv_bfloat16 *)dZ, dW, db,
        4000000000LL);
    return launched("conv3x3_wgrad_tc_kernel");
}

int cnn_conv3x3_tc(const void *X, int N, int H, int W, int dil, const void *Wt,
                   const float *bias, int relu, void *Y, cudaStream_t stream) {
    if (dil < 1 || dil > kTcHalo || W < 1 || H < 1 || N < 1)
        return set_error(FHTDP_EINVAL, "conv3x3: dilation 1..8 and a non-empty image");
    // persistent CTAs: the weights and two stages (73.7 KB), three per SM
    const size_t smem = (size_t)kBBytes + 2 * kABytes;
    // set on every call: the attribute belongs to the current device
    int st = cuda_status(cudaFuncSetAttribute(relu ? conv3x3_tc_persist_kernel<true>
                                                   : conv3x3_tc_persist_kernel<false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem),
                         "cudaFuncSetAttribute");
    if (st) return st;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long units = (long long)N * H * ((W + kTcM - 1) / kTcM);
    const long long grid = std::min<long long>(units, 3LL * (sms > 0 ? sms : 152));
    const long long wait = 4000000000LL;   // about two seconds
    if (relu)
        conv3x3_tc_persist_kernel<true><<<(unsigned)grid, kTcThreads, smem, stream>>>(
            (const __nv_bfloat16 *)X, N, H, W, dil, (const __nv_bfloat16 *)Wt, bias,
            (__nv_bfloat16 *)Y, wait);
    else
        conv3x3_tc_persist_kernel<false><<<(unsigned)grid, kTcThreads, smem, stream>>>(
            (const __nv_bfloat16 *)X, N, H, W, dil, (const __nv_bfloat16 *)Wt, bias,
            (__nv_bfloat16 *)Y, wait);
    return launched("conv3x3_tc_persist_kernel");
}

int cnn_tc_status(int clear) {
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_conv_tc_status, sizeof(int));
    if (e != cudaSuccess) return cuda_status(e, "cudaMemcpyFromSymbol");
    if (clear) {
        const int z = 0;
        e = cudaMemcpyToSymbol(g_conv_tc_status, &z, sizeof(int));
        if (e != cudaSuccess) return cuda_status(e, "cudaMemcpyToSymbol");
    }
    return v;
}

}  // namespace fhtdp
