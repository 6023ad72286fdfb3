// Fused detection engine: band FHT + bend-limited DP + read-back in one
// persistent kernel.
//
// Work items are (image, band, column tile) taken from a device-side queue
// in which every item comes after the band+1 tiles it depends on.  An item
//   1. computes the Hough values of its band for its T output columns in
//      shared memory (Sec. 2.1): the band strip with its n-1 column halo is
//      loaded, and the log2(n) dyadic levels are merged in place;
//   2. waits until the three tiles of band+1 that it depends on have
//      published their window maxima (bounded spin, see wait_flag);
//   3. forms V_b(x, e) = H_b(x, e) + M_{b+1}(x + e, e) (Eqs. 3-4) and the
//      bend-window maxima M_b(x, c) = max_{|e - c| <= B} V_b(x, e)
//      (Sec. 2.3, RangeMaxQ) with the van Herk / Gil-Werman block method,
//      carrying the argmax in the low bits of an integer key; it writes M_b
//      (to an L2-resident ping-pong buffer, skewed so that the consumer's
//      gather M_b(x + d, d) is a contiguous row read) and the argmax byte
//      bp_b(x, c), then publishes its flag;
//   4. on band 0 it reduces V_0 to the lexicographically smallest argmax
//      (main problem, steps 2-3); the last band-0 tile of an image reads the
//      polyline back through bp (Eq. 5).
// The Hough images and the DP values never reach global memory.
//
// Pixel types: uint8 images keep both slope halves of a Hough value in one
// 32-bit word (two 16-bit lanes: sums of at most 128 uint8 pixels fit), so
// one shared-memory access and one integer add serve both halves.  The "-"
// half is computed on the mirrored strip, so both halves use the same
// merge.  int32 and float images run the halves one after the other.
#include <algorithm>
#include <climits>
#include <cstddef>
#include <new>
#include <type_traits>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "engine.cuh"

namespace fhtdp {
namespace {

constexpr int kThreads = 512;
constexpr int kTile = 128;             // output columns of one item
constexpr int kQ = kThreads / kTile;   // threads sharing a column in the DP
// The uint8 engine adds a fifth warpgroup whose first warp runs the control
// of the work items (queue, dependency flags, copies, publication) so that
// its waits stay off the compute warps' path; the other three warps exit.
constexpr int kWsThreads = kThreads + 128;
constexpr int kCtlSync = kThreads + 32;   // compute threads + the control warp
// Named barriers: 1 among the compute threads; 2..5 between them and the
// control warp (compute threads arrive, the control warp waits, or back).
constexpr int kBarCompute = 1, kBarFhtDone = 2, kBarHcFree = 3, kBarWinDone = 4, kBarNext = 5;
constexpr int kMaxBandFused = 128;     // band heights handled by the fused kernel
constexpr int kMOff = 128;             // column offset of the skewed M layout
constexpr int kPad = 16;               // dead rows around V (uint8 path)
constexpr int kFastB = 16;             // largest bend kept entirely in registers
// 256-row bands: DP items take 64 columns; V of such an item ((511 + 2 kPad)
// rows of 64 words) is followed by the window's suffix maxima.
constexpr int kTile256 = 64;
constexpr int kDp256SOff = (511 + 2 * kPad) * kTile256 * 4;
// Margins of an h256 row (elements): the DP items read up to 128 columns
// left of column 0 and up to 196 right of the last tile; the row starts at
// kH256Left so that both stay inside it.
constexpr int kH256Left = 136, kH256Right = 200;
// M tile of a 256-row-band DP item: 511 rows in 7 copies of 73.
constexpr int kMBox256 = 73;
// After a copy wait gives up, the last bounded wait for that copy to land
// before its shared memory is reused (about four seconds).
constexpr long long kDrainCycles = 8000000000LL;

struct ImgDesc {
    CUtensorMap tmap;         // 2-D map of the image (uint8 images), box 128 x n
    CUtensorMap mtmap;        // 2-D map of both M buffers, [2D][mpitch] int32, box 128 x D
    int use_tma;              // strip loads through tmap
    int use_mtma;             // M tiles through mtmap (uint8 images)
    const void *img;
    long long pitch;          // row stride in elements
    int h, w, k, n, log2n, B, tiles;
    int tw;                   // column tile width of its work items (uint8: 64, 128 or 256)
    int depth;                // uint8: FHT levels done in registers before the merges (2 or 3)
    long long item0;          // first work item of this image
    void *mbuf[2];            // ping-pong window maxima, [D][mpitch] of Acc
    int mpitch;
    uint8_t *bp;              // argmax index of each window, see bp_byte
    int *flags;               // [k][tiles] publication flags
    unsigned long long *best; // lexicographic argmax key of V_0
    int *done;                // band-0 tiles finished
    int32_t *x_out, *d_out;
    void *score_out;
    const int32_t *win;       // optional [k][2]: allowed displacements of each band
    // uint8 images with 256-row bands (kind 1): each band's Hough values are
    // built from the FHTs of its two 128-row halves (half-band items, stored
    // in h256), merged by the last dyadic level inside the DP items.
    int kind;                 // 0: bands of at most 128 rows; 1: 256-row bands
    int ftiles;               // half-band FHT tiles of 128 columns
    int hpitch;               // row pitch of h256 in elements
    uint16_t *h256;           // [k][2 halves][2 signs][128 shifts][hpitch], see h256_row
    int *fflags;              // [k][2][ftiles] publication flags of the half-band items
                              // (int32 / float images: [k][ftiles], their FHT items)
    int moff;                 // column offset of the skewed M layout
    // int32 / float images (kind 2): Hough rows of every band stored by the
    // FHT items, [k][2 signs][n][hwpitch] of 4-byte values; `tmap` then
    // describes them for the DP items' TMA copies (boxes of 32 x n).
    void *hw;
    int hwpitch;
    // Optional device flag: when it reads 0 at the launch, every item of the
    // image is skipped (the learned proposal's fallback run only redoes the
    // images that need the full DP).
    const int32_t *enable;
    // Subproblems 2-3 (uint8 images, bands of at most 128 rows): when mask1 >
    // 0, every state of band mask1 - 1 whose vertex on the point's border is
    // not mask_x is dead: the link's start x (mask_end = 0, the point on the
    // band's upper border) or its end x + d (mask_end = 1, the image's bottom
    // border).
    int mask1, mask_x, mask_end;
};

// Backpointers: per band, ceil(D/4) groups of w 32-bit words; byte (e & 3)
// of word (band, e >> 2, x) is the argmax index of the window of state
// (x, e), e = c + n - 1.  Four displacements of a column share a word, so
// the window, which runs along e for a fixed x, stores a word per four.
__host__ __device__ inline int bp_groups(int n) { return (2 * n - 1 + 3) / 4; }
__device__ __forceinline__ size_t bp_byte(const ImgDesc &im, int band, int e, int x) {
    return (((size_t)band * bp_groups(im.n) + (e >> 2)) * im.w + x) * 4 + (e & 3);
}

struct Ctl {
    int queue;   // next work item
    int status;  // FHTDP_OK or FHTDP_ETIMEOUT
    int pad[62];
};

// One work item of a batch: image index, band, column tile, and the image's
// band height n with bit 16 set when its strips go through TMA.
struct Item {
    int image, band, tile, nflags;
};

struct LaunchArgs {
    ImgDesc one;              // single-image launches
    const ImgDesc *many;      // batched launches (device array), or null
    const Item *order;        // batched launches: the queue, item by item
    int count;
    long long items;
    Ctl *ctl;
    long long wait_cycles;
    // Fault injection for tests (fhtdp_debug_inject): the tile (band, tile)
    // of the first image never publishes; -1 disables.
    int skip_band, skip_tile;
    // int32 / float images, one image: with use_table the bend-angle windows
    // of Sec. 2.3 (Eqs. 6-7) replace |e - d| <= B, e in [tab.lo[d + n - 1],
    // tab.hi[d + n - 1]].  The DP items answer them from maxima of fixed
    // half-width B0 (every window that no end of the displacement range
    // clips is at least 2 B0 + 1 long), with wpad dead rows above and below V.
    int use_table, B0, wpad;
    WindowTable tab;
};

// ---------------------------------------------------------------------------
// Value <-> order-preserving integers.
__device__ __forceinline__ uint32_t ord32(int32_t v) { return (uint32_t)v ^ 0x80000000u; }
__device__ __forceinline__ uint32_t ord32(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
template <typename Acc>
__device__ __forceinline__ Acc from_ord32(uint32_t o);
template <>
__device__ __forceinline__ int32_t from_ord32<int32_t>(uint32_t o) {
    return (int32_t)(o ^ 0x80000000u);
}
template <>
__device__ __forceinline__ float from_ord32<float>(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

template <typename W>
__device__ __forceinline__ W from_bits(uint32_t b);
template <>
__device__ __forceinline__ uint32_t from_bits<uint32_t>(uint32_t b) { return b; }
template <>
__device__ __forceinline__ int32_t from_bits<int32_t>(uint32_t b) { return (int32_t)b; }
template <>
__device__ __forceinline__ float from_bits<float>(uint32_t b) { return __uint_as_float(b); }
__device__ __forceinline__ uint32_t to_bits(uint32_t v) { return v; }
__device__ __forceinline__ uint32_t to_bits(int32_t v) { return (uint32_t)v; }
__device__ __forceinline__ uint32_t to_bits(float v) { return __float_as_uint(v); }

// Window keys: a value and its displacement index e + n - 1 (< 512) in one
// integer whose maximum is the largest value with the smallest index.
template <typename Acc, typename Key>
struct KeyOps;
template <>
struct KeyOps<int32_t, int32_t> {   // non-negative values below 2^22; dead keys < 0
    __device__ static int32_t dead() { return INT32_MIN; }
    __device__ static int32_t make(int32_t v, int e) { return (v << 9) | (511 - e); }
    __device__ static int32_t value(int32_t k) { return k >> 9; }
    __device__ static int index(int32_t k) { return 511 - (k & 511); }
};
template <typename Acc>
struct KeyOps<Acc, long long> {
    __device__ static long long dead() { return LLONG_MIN; }
    __device__ static long long make(Acc v, int e) {
        int32_t so = (int32_t)(ord32(v) ^ 0x80000000u);
        return ((long long)so << 9) | (511 - e);
    }
    __device__ static Acc value(long long k) {
        return from_ord32<Acc>((uint32_t)(int32_t)(k >> 9) ^ 0x80000000u);
    }
    __device__ static int index(long long k) { return 511 - (int)(k & 511); }
};

template <typename T>
__device__ __forceinline__ T kmax(T a, T b) {
    return a > b ? a : b;
}
__device__ __forceinline__ float kmax(float a, float b) { return fmaxf(a, b); }

__device__ __forceinline__ int brev(int r, int bits) {
    return bits ? (int)(__brev((unsigned)r) >> (32 - bits)) : 0;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
// Barrier of the kThreads compute threads (every thread of the 512-thread
// kernel; the compute warps of the uint8 kernel), or of NT threads.
template <int NT = kThreads>
__device__ __forceinline__ void csync() {
    asm volatile("bar.sync %0, %1;" ::"n"(kBarCompute), "n"(NT) : "memory");
}
__device__ __forceinline__ void nb_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void nb_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Bounded wait on a publication flag: gives up after `limit` cycles, or at
// once when another wait of this launch has already given up.
// A hint to bring the 128-byte line holding p into L2 (callers pass only
// lines that hold bytes of their buffers).
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ bool wait_flag(const int *flag, const Ctl *ctl, long long limit) {
    long long t0 = clock64();
    while (ld_acquire(flag) == 0) {
        if (*(volatile const int *)&ctl->status != FHTDP_OK) return false;
        if (clock64() - t0 > limit) return false;
        __nanosleep(100);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Tensor-memory-access (TMA) copies into shared memory, completed on an
// mbarrier.  Every wait is bounded like the flag waits.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(
            smem_addr(bar)),
        "r"(bytes)
        : "memory");
}
// Waits for the phase `parity` of `bar` to complete; false after `limit` cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
            "selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Orders global data observed through the generic proxy (M published by
// other CTAs) before this thread's later TMA reads of it.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
// 2-D tile (x, y) of a tensor map into shared memory.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
// Per-CTA state of the asynchronous copies and of the queue: the next work
// item is taken before the current one finishes, so that its band strip can
// be copied while the current item computes its window maxima.
// The item the control warp hands to the compute warps of the uint8 engine.
struct WsSlot {
    long long item;
    const ImgDesc *im;
    int band, tile, prefetched, T, kind;
};

// Work-item kinds (queue-entry bits 19-20).
constexpr int kItemBand = 0;    // FHT + DP of a tile of a band of at most 128 rows
constexpr int kItemHalf0 = 1;   // FHT of the top 128-row half of a 256-row band
constexpr int kItemHalf1 = 2;   // FHT of the bottom half
constexpr int kItemDp256 = 3;   // last FHT level + DP of a 64-column tile of a 256-row band

struct NextItem {
    long long item;
    int prefetched;   // its strip copy has been issued on the strip barrier
    int pad;
    Item it;          // its order entry (batches), copied by cp.async
};
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}
struct Pipe {
    uint64_t *bar;        // strip barrier
    uint32_t phase;       // parity of its next completion
    uint64_t *mbar;       // M tile barrier
    uint32_t mphase;      // parity of its next completion
    NextItem *next;       // shared: the CTA's next item
};

// Thread 0: records the item taken from the queue and starts copying its
// order entry (completed by cp_async_wait_all before anyone reads it).
__device__ __forceinline__ void stage_next(const LaunchArgs &args, NextItem *next,
                                           long long item) {
    next->item = item;
    next->prefetched = 0;
    if (args.many && item < args.items) cp_async16(&next->it, &args.order[item]);
}
// The staged item (item < items).
__device__ __forceinline__ void decode_staged(const LaunchArgs &args, const NextItem &nx,
                                              const ImgDesc **imp, int *band, int *tile) {
    if (args.many) {
        *imp = &args.many[nx.it.image];
        *band = nx.it.band;
        *tile = nx.it.tile;
    } else {
        *imp = &args.one;
        *band = args.one.k - 1 - (int)(nx.item / args.one.tiles);
        *tile = (int)(nx.item % args.one.tiles);
    }
}

__device__ __forceinline__ uint32_t pix_u8(const uint8_t *row, int col, int w) {
    return (col >= 0 && col < w) ? (uint32_t)row[col] : 0u;
}
template <typename In>
__device__ __forceinline__ In pix(const In *row, int col, int w) {
    return (col >= 0 && col < w) ? row[col] : In(0);
}

// ---------------------------------------------------------------------------
// Shared-memory FHT of one band strip (Sec. 2.1).  F holds n rows of `pitch`
// words (pitch >= T + n + 8, a multiple of 4).  Row y of the strip is loaded
// into row y; after the level of m-row sub-bands, row j*m + brev(s) holds
// shift s of sub-band j, so at the end row brev(s) holds the Hough row of
// shift s.  Merging at level m pairs row A = j*m + r with row B = j*m + m/2 + r
// (r = brev(s') over log2(m)-1 bits):
//   A <- A(u) + B(u + s'),   B <- A(u) + B(u + s' + 1)
// i.e. out(u, 2s') and out(u, 2s'+1) of the recursion.  A warp owns a row
// pair and sweeps its columns left to right, 128 at a time (4 per lane, with
// 16-byte shared loads and stores; the shift modulo 4 is warp-uniform and
// selects a fixed register pattern): column u of row B is only read by
// columns <= u, so the update is in place.  Columns past the level's valid
// width are computed from stale words and are never read by valid ones.
template <typename W, int Q>
__device__ __forceinline__ void merge4(const uint4 &a4, const uint4 &b0, const uint4 &b1,
                                       uint4 &oa, uint4 &ob) {
    const W a[4] = {from_bits<W>(a4.x), from_bits<W>(a4.y), from_bits<W>(a4.z),
                    from_bits<W>(a4.w)};
    const W b[8] = {from_bits<W>(b0.x), from_bits<W>(b0.y), from_bits<W>(b0.z),
                    from_bits<W>(b0.w), from_bits<W>(b1.x), from_bits<W>(b1.y),
                    from_bits<W>(b1.z), from_bits<W>(b1.w)};
    oa.x = to_bits(a[0] + b[Q + 0]);
    oa.y = to_bits(a[1] + b[Q + 1]);
    oa.z = to_bits(a[2] + b[Q + 2]);
    oa.w = to_bits(a[3] + b[Q + 3]);
    ob.x = to_bits(a[0] + b[Q + 1]);
    ob.y = to_bits(a[1] + b[Q + 2]);
    ob.z = to_bits(a[2] + b[Q + 3]);
    ob.w = to_bits(a[3] + b[Q + 4]);
}

// With `out`, the last level writes shift s to row s of out (pitch T)
// instead of in place.
// NT threads take part; `out` rows are opitch words apart (default T).
template <typename W, int NT = kThreads>
__device__ void fht_levels(W *F, int pitch, int n, int log2n, int T, int first = 1,
                           W *out = nullptr, int opitch = 0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = NT / 32;
    if (!opitch) opitch = T;
    for (int l = first; l <= log2n; ++l) {
        const int m = 1 << l, half = m >> 1;
        const int width = T + n - m;
        const bool to_out = out && l == log2n;
        for (int p = warp; p < n / 2; p += nwarps) {
            const int j = p >> (l - 1), r = p & (half - 1);
            const int sp = brev(r, l - 1);
            const int q = sp & 3;   // warp-uniform
            W *A = F + (size_t)(j * m + r) * pitch;
            W *Brow = F + (size_t)(j * m + half + r) * pitch;
            const W *Bq = Brow + (sp - q);
            for (int u0 = 0; u0 < width; u0 += 128) {
                const int u = u0 + 4 * lane;
                const bool live = u < width;
                uint4 oa = make_uint4(0, 0, 0, 0), ob = oa;
                if (live) {
                    const uint4 a4 = *(const uint4 *)&A[u];
                    const uint4 b0 = *(const uint4 *)&Bq[u];
                    const uint4 b1 = *(const uint4 *)&Bq[u + 4];
                    switch (q) {
                        case 0: merge4<W, 0>(a4, b0, b1, oa, ob); break;
                        case 1: merge4<W, 1>(a4, b0, b1, oa, ob); break;
                        case 2: merge4<W, 2>(a4, b0, b1, oa, ob); break;
                        default: merge4<W, 3>(a4, b0, b1, oa, ob); break;
                    }
                }
                if (to_out) {   // one sub-band: shifts 2sp, 2sp+1 at width T
                    if (live) {
                        *(uint4 *)&out[(size_t)(2 * sp) * opitch + u] = oa;
                        *(uint4 *)&out[(size_t)(2 * sp + 1) * opitch + u] = ob;
                    }
                    continue;
                }
                __syncwarp();
                if (live) {
                    *(uint4 *)&A[u] = oa;
                    *(uint4 *)&Brow[u] = ob;
                }
                __syncwarp();
            }
        }
        csync<NT>();
    }
}

// Two dyadic levels in one shared-memory pass: four consecutive sub-bands
// J0..J3 of m rows, all at shift q, give the shifts 4q..4q+3 of the merged
// sub-band of 4m rows.  With A = (J0, J1) and B = (J2, J3) merged first,
//   out(u, 4q+0) = [J0(u) + J1(u+q)]   + [J2(u+2q)   + J3(u+3q)]
//   out(u, 4q+1) = [J0(u) + J1(u+q)]   + [J2(u+2q+1) + J3(u+3q+1)]
//   out(u, 4q+2) = [J0(u) + J1(u+q+1)] + [J2(u+2q+1) + J3(u+3q+2)]
//   out(u, 4q+3) = [J0(u) + J1(u+q+1)] + [J2(u+2q+2) + J3(u+3q+3)]
// (the same summation tree as two radix-2 levels).  Shift 4q+r goes to the
// row of J_{brev2(r)} at the same in-sub-band slot, so the pass is in place
// under the same left-to-right sweep rule.  O1..O3 are the word offsets of
// u+q, u+2q, u+3q inside their 16-byte-aligned loads.
template <typename W, int O1, int O2, int O3>
__device__ __forceinline__ void merge4x4(const uint4 &j0, const uint4 *j1, const uint4 *j2,
                                         const uint4 *j3, uint4 *out) {
    const W a[4] = {from_bits<W>(j0.x), from_bits<W>(j0.y), from_bits<W>(j0.z),
                    from_bits<W>(j0.w)};
    W b1[8], b2[8], b3[12];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        b1[4 * k + 0] = from_bits<W>(j1[k].x);
        b1[4 * k + 1] = from_bits<W>(j1[k].y);
        b1[4 * k + 2] = from_bits<W>(j1[k].z);
        b1[4 * k + 3] = from_bits<W>(j1[k].w);
        b2[4 * k + 0] = from_bits<W>(j2[k].x);
        b2[4 * k + 1] = from_bits<W>(j2[k].y);
        b2[4 * k + 2] = from_bits<W>(j2[k].z);
        b2[4 * k + 3] = from_bits<W>(j2[k].w);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        b3[4 * k + 0] = from_bits<W>(j3[k].x);
        b3[4 * k + 1] = from_bits<W>(j3[k].y);
        b3[4 * k + 2] = from_bits<W>(j3[k].z);
        b3[4 * k + 3] = from_bits<W>(j3[k].w);
    }
    uint32_t o[4][4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const W A0 = a[t] + b1[O1 + t], A1 = a[t] + b1[O1 + t + 1];
        const W B0 = b2[O2 + t] + b3[O3 + t];
        const W B1 = b2[O2 + t + 1] + b3[O3 + t + 1];
        const W B2 = b2[O2 + t + 1] + b3[O3 + t + 2];
        const W B3 = b2[O2 + t + 2] + b3[O3 + t + 3];
        o[0][t] = to_bits(A0 + B0);
        o[1][t] = to_bits(A0 + B1);
        o[2][t] = to_bits(A1 + B2);
        o[3][t] = to_bits(A1 + B3);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) out[r] = make_uint4(o[r][0], o[r][1], o[r][2], o[r][3]);
}

// Levels l+1 and l+2 (sub-bands of m = 2^l rows merged into 4m rows).  With
// `out` (only when 4m = n) shift s goes to row s of out (pitch T).
template <typename W, int NT = kThreads>
__device__ void fht_radix4(W *F, int pitch, int n, int l, int T, W *out = nullptr,
                           int opitch = 0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = NT / 32;
    if (!opitch) opitch = T;
    const int m = 1 << l;
    const int width = T + n - 4 * m;
    for (int p = warp; p < n / 4; p += nwarps) {
        const int g4 = p >> l, r = p & (m - 1);
        const int q = brev(r, l);
        const int o = q & 3;   // warp-uniform
        W *J[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) J[t] = F + (size_t)((4 * g4 + t) * m + r) * pitch;
        const W *B1 = J[1] + (q - (q & 3));
        const W *B2 = J[2] + (2 * q - ((2 * q) & 3));
        const W *B3 = J[3] + (3 * q - ((3 * q) & 3));
        for (int u0 = 0; u0 < width; u0 += 128) {
            const int u = u0 + 4 * lane;
            const bool live = u < width;
            uint4 o4[4];
            if (live) {
                const uint4 j0 = *(const uint4 *)&J[0][u];
                const uint4 j1[2] = {*(const uint4 *)&B1[u], *(const uint4 *)&B1[u + 4]};
                const uint4 j2[2] = {*(const uint4 *)&B2[u], *(const uint4 *)&B2[u + 4]};
                const uint4 j3[3] = {*(const uint4 *)&B3[u], *(const uint4 *)&B3[u + 4],
                                     *(const uint4 *)&B3[u + 8]};
                switch (o) {
                    case 0: merge4x4<W, 0, 0, 0>(j0, j1, j2, j3, o4); break;
                    case 1: merge4x4<W, 1, 2, 3>(j0, j1, j2, j3, o4); break;
                    case 2: merge4x4<W, 2, 0, 2>(j0, j1, j2, j3, o4); break;
                    default: merge4x4<W, 3, 2, 1>(j0, j1, j2, j3, o4); break;
                }
            }
            if (out) {
                if (live) {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        *(uint4 *)&out[(size_t)(4 * q + t) * opitch + u] = o4[t];
                }
                continue;
            }
            __syncwarp();
            if (live) {
                *(uint4 *)&J[0][u] = o4[0];   // shift 4q+0 -> row of J0
                *(uint4 *)&J[2][u] = o4[1];   // shift 4q+1 -> row of J2 (brev2(1) = 2)
                *(uint4 *)&J[1][u] = o4[2];   // shift 4q+2 -> row of J1
                *(uint4 *)&J[3][u] = o4[3];   // shift 4q+3 -> row of J3
            }
            __syncwarp();
        }
    }
    csync<NT>();
}

// All levels from `first` (sub-bands of 2^(first-1) rows already merged),
// two at a time where possible.  With `out` the last level writes shift s to
// row s of out; returns whether there was a level to do so.
template <typename W, int NT = kThreads>
__device__ bool fht_merge(W *F, int pitch, int n, int log2n, int T, int first,
                          W *out = nullptr, int opitch = 0) {
    int l = first - 1;   // current sub-band size 2^l
    while (l + 2 <= log2n) {
        fht_radix4<W, NT>(F, pitch, n, l, T, l + 2 == log2n ? out : nullptr, opitch);
        l += 2;
    }
    if (l < log2n) fht_levels<W, NT>(F, pitch, n, log2n, T, l + 1, out, opitch);
    return first <= log2n;
}

// ---------------------------------------------------------------------------
// Window maxima of one column (Sec. 2.3): M(c) = max_{|e-c|<=B} V(e) for c in
// [c0, c1], as keys carrying the argmax.  Blocks of length L = 2B+1 start at
// c0 - B; M(c0 + (q-1)L + i) = max(S_{q-1}[i], G_q[i-1]) with S the in-block
// suffix maximum and G the in-block prefix maximum (van Herk / Gil-Werman),
// or S_{q-1}[0] for i = 0.  Register version: L <= LMAX (L == LMAX when
// kExact), every value of the column range read once from shared memory.
template <int LMAX, bool kExact, typename Key, typename VGet, typename Emit>
__device__ __forceinline__ void window_regs(int c0, int c1, int B, Key dead, VGet vkey,
                                            Emit emit) {
    const int L = kExact ? LMAX : 2 * B + 1;
    Key S[LMAX], Vb[LMAX];
    const int a0 = c0 - B;
#pragma unroll
    for (int i = 0; i < LMAX; ++i) Vb[i] = (kExact || i < L) ? vkey(a0 + i) : dead;
    Key run = dead;
#pragma unroll
    for (int i = LMAX - 1; i >= 0; --i) {
        if (kExact || i < L) run = kmax(run, Vb[i]);
        S[i] = run;
    }
    for (int c = c0, base = a0 + L; c <= c1; c += L, base += L) {
        Key G = dead;
#pragma unroll
        for (int i = 0; i < LMAX; ++i) {
            if (kExact || i < L) {
                const Key v = vkey(base + i);
                Vb[i] = v;
                const Key m = i == 0 ? S[0] : kmax(S[i], G);
                G = kmax(G, v);
                if (c + i <= c1) emit(c + i, m);
            }
        }
        run = dead;
#pragma unroll
        for (int i = LMAX - 1; i >= 0; --i) {
            if (kExact || i < L) run = kmax(run, Vb[i]);
            S[i] = run;
        }
    }
}

// The register window of the uint8 path for L = 2B+1 in {9, 17, 25, 33}
// (L = 1 mod 4) over at most 64 displacements: outputs j = c - ca, ca at a
// bp word boundary.  kcol[c * kTile] is the V key of displacement c (dead
// pad rows outside [lo, hi]); output j stores M' = key & ~511 to
// mcol[j * mstride] and its index byte into bp word bcol[(j >> 2) * bstride].
// The blocks are unrolled, so each byte's place in its word is a constant.
template <int L>
__device__ __forceinline__ void window_u8(int ca, int c1, const int32_t *kcol, int32_t *mcol,
                                          int mstride, uint32_t *bcol, int bstride) {
    constexpr int B = (L - 1) / 2;
    constexpr int NB = (64 + L - 1) / L;
    static_assert(L % 4 == 1, "block starts must keep the byte phase");
    int32_t S[L], Vb[L];
    const int32_t *kp = kcol + (ca - B) * kTile;
#pragma unroll
    for (int i = 0; i < L; ++i) Vb[i] = kp[i * kTile];
    int32_t run = INT32_MIN;
#pragma unroll
    for (int i = L - 1; i >= 0; --i) {
        run = max(run, Vb[i]);
        S[i] = run;
    }
    const int last = c1 - ca;
    uint32_t word = 0;
    int32_t *mp = mcol;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        if (k * L > last) break;
        const int32_t *vp = kcol + (ca + k * L + B + 1) * kTile;
        int32_t G = INT32_MIN;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            const int j = k * L + i;
            const int32_t v = vp[i * kTile];
            Vb[i] = v;
            const int32_t m = i == 0 ? S[0] : max(S[i], G);
            G = max(G, v);
            if (j <= last) {
                *mp = m & ~511;
                const uint32_t b = ~(uint32_t)m & 0xffu;
                word = (j & 3) == 0 ? b : word | (b << (8 * (j & 3)));
                if ((j & 3) == 3) bcol[(j >> 2) * bstride] = word;
            }
            mp += mstride;
        }
        if (k + 1 < NB) {
            run = INT32_MIN;
#pragma unroll
            for (int i = L - 1; i >= 0; --i) {
                run = max(run, Vb[i]);
                S[i] = run;
            }
        }
    }
    if ((last & 3) != 3) bcol[(last >> 2) * bstride] = word;
}

// Register version for L = 2B+1 <= LMAX that keeps only the suffix maxima S
// in registers: each block's values are read once for the prefix pass and
// once more for the next block's suffix maxima (for long windows, where
// holding the block's values too would not fit).
template <int LMAX, typename Key, typename VGet, typename Emit>
__device__ __forceinline__ void window_reread(int c0, int c1, int B, Key dead, VGet vkey,
                                              Emit emit) {
    const int L = 2 * B + 1;
    Key S[LMAX];
    int a = c0 - B;   // first input of the current block
    Key run = dead;
#pragma unroll
    for (int i = LMAX - 1; i >= 0; --i) {
        if (i < L) run = kmax(run, vkey(a + i));
        S[i] = run;
    }
    for (int c = c0; c <= c1; c += L) {
        a += L;
        Key G = dead;
#pragma unroll
        for (int i = 0; i < LMAX; ++i) {
            if (i < L) {
                const Key v = vkey(a + i);
                const Key m = i == 0 ? S[0] : kmax(S[i], G);
                G = kmax(G, v);
                if (c + i <= c1) emit(c + i, m);
            }
        }
        if (c + L <= c1) {
            run = dead;
#pragma unroll
            for (int i = LMAX - 1; i >= 0; --i) {
                if (i < L) run = kmax(run, vkey(a + i));
                S[i] = run;
            }
        }
    }
}

// Window maxima of the 32 displacements [c0, c0 + 31] for 16 <= B <= 32
// (L = 2B + 1 > 32), one block pair of the van Herk / Gil-Werman scheme:
// M(c0 + i) = max(S[i], G(i)) with S[i] the maximum of V over
// [c0 - B + i, c0 + B] and G(i) that over [c0 + B + 1, c0 + B + i] (empty for
// i = 0).  Only S[0..31] is kept (in registers).  Output i < count stores M'
// (the key with its index bits cleared) to mcol[i * mstride] and packs its
// argmax byte (the index modulo 256) into the word bcol[(i >> 2) * bstride].
template <typename VGet>
__device__ __forceinline__ void window_span32(int c0, int count, int B, VGet vkey,
                                              int32_t *mcol, int mstride, uint32_t *bcol,
                                              int bstride) {
    const int L = 2 * B + 1;
    int32_t S[32];
    int32_t run = INT32_MIN;
    const int a = c0 - B;
#pragma unroll
    for (int j = 64; j >= 0; --j) {
        if (j < L) run = max(run, vkey(a + j));
        if (j < 32) S[j] = run;
    }
    int32_t G = INT32_MIN;
    uint32_t word = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int32_t m = max(S[i], G);
        G = max(G, vkey(c0 + B + 1 + i));
        if (i < count) mcol[i * mstride] = m & ~511;
        const uint32_t b = ~(uint32_t)m & 0xffu;
        word = (i & 3) == 0 ? b : word | (b << (8 * (i & 3)));
        if ((i & 3) == 3) bcol[(i >> 2) * bstride] = word;
    }
}

// Window maxima of the NOUT displacements [c0, c0 + NOUT - 1] for windows
// of L = 2B + 1 >= NOUT (any B beyond that), one block pair of the van Herk /
// Gil-Werman scheme: S[i] (registers) is the maximum over [c0 - B + i, c0 + B]
// and G that over [c0 + B + 1, c0 + B + i]; output i < count goes to emit(i, m).
template <int NOUT, typename Key, typename VGet, typename Emit>
__device__ __forceinline__ void window_span(int c0, int count, int B, Key dead, VGet vkey,
                                            Emit emit) {
    const int L = 2 * B + 1;
    const int a = c0 - B;
    Key run = dead;
    int j = L - 1;
    // the part of the block beyond the first NOUT values: 8 loads at a time
    for (; j - 7 >= NOUT; j -= 8) {
        Key k[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) k[i] = vkey(a + j - i);
#pragma unroll
        for (int i = 0; i < 8; i += 2) k[i] = kmax(k[i], k[i + 1]);
        run = kmax(run, kmax(kmax(k[0], k[2]), kmax(k[4], k[6])));
    }
    for (; j >= NOUT; --j) run = kmax(run, vkey(a + j));
    Key S[NOUT];
#pragma unroll
    for (int jj = NOUT - 1; jj >= 0; --jj) {
        run = kmax(run, vkey(a + jj));
        S[jj] = run;
    }
    Key G = dead;
#pragma unroll
    for (int i = 0; i < NOUT; ++i) {
        const Key m = kmax(S[i], G);
        G = kmax(G, vkey(c0 + B + 1 + i));
        if (i < count) emit(i, m);
    }
}

// Two-pass version for any L: pass 1 stores the in-block suffix maxima
// S(e), e in [c0-B, c1-B], through sput/sget; pass 2 runs the in-block prefix
// maximum G(c+B) and combines.  Blocks are aligned at `a` (a <= c0 - B).
template <typename Key, typename VGet, typename SPut, typename SGet, typename Emit>
__device__ __forceinline__ void window_two_pass(int c0, int c1, int B, int a, int lo, int hi,
                                                Key dead, VGet vkey, SPut sput, SGet sget,
                                                Emit emit) {
    const int L = 2 * B + 1;
    int e = a + ((c1 - B - a) / L + 1) * L - 1;   // end of the block of c1-B
    if (e > hi) e = hi;
    int pos = (e - a) % L;
    Key run = dead;
    for (; e >= c0 - B; --e) {
        const Key v = vkey(e);
        run = pos == L - 1 ? v : kmax(run, v);
        if (e <= c1 - B) sput(e, run);
        pos = pos == 0 ? L - 1 : pos - 1;
    }
    int g = a + ((c0 + B - a) / L) * L;   // start of the block of c0+B
    if (g < lo) g = lo;
    pos = (g - a) % L;
    Key gr = dead;
    for (; g <= c1 + B; ++g) {
        const Key v = vkey(g);
        gr = pos == 0 ? v : kmax(gr, v);
        pos = pos == L - 1 ? 0 : pos + 1;
        if (g >= c0 + B) emit(g - B, kmax(sget(g - 2 * B), gr));
    }
}

// Allowed displacements of a band: [lo, hi] (the whole range unless the
// image carries windows, as for the pruned DP of the learned proposal).
__device__ __forceinline__ void band_window(const ImgDesc &im, int band, int *lo, int *hi) {
    int a = -(im.n - 1), b = im.n - 1;
    if (im.win) {
        a = max(a, __ldg(im.win + 2 * band));
        b = min(b, __ldg(im.win + 2 * band + 1));
    }
    *lo = a;
    *hi = b;
}

// Eq. 5: the polyline from the best top point, one backpointer per band.
template <typename Acc>
__device__ void readback(const ImgDesc &im, const LaunchArgs &args) {
    const int n = im.n;
    __threadfence();
    const unsigned long long key = atomicAdd(im.best, 0ull);
    if (key == 0) {   // no admissible polyline inside the windows
        *(Acc *)im.score_out = Dead<Acc>::value();
        for (int i = 0; i <= im.k; ++i) im.x_out[i] = -1;
        for (int i = 0; i < im.k; ++i) im.d_out[i] = 0;
        return;
    }
    const unsigned lin = 0xffffffffu - (unsigned)(key & 0xffffffffu);
    int xx = (int)(lin >> 9), d = (int)(lin & 511) - (n - 1);
    im.x_out[0] = xx;
    im.d_out[0] = d;
    *(Acc *)im.score_out = from_ord32<Acc>((uint32_t)(key >> 32));
    for (int i = 1; i < im.k; ++i) {
        xx += d;
        // Only reachable with inconsistent DP data (a wait gave up): stop
        // instead of reading outside bp.
        if (xx < 0 || xx >= im.w || d < -(n - 1) || d > n - 1) {
            atomicExch(&args.ctl->status, FHTDP_ETIMEOUT);
            return;
        }
        int e = __ldcg(im.bp + bp_byte(im, i, d + n - 1, xx));
        // 256-row bands: the byte holds the index modulo 256; the window
        // [c - B, c + B] (B <= 127) around c = d + n - 1 has one index per residue.
        if (n > 128) {
            const int lo = d + n - 1 - im.B;
            e = lo + ((e - lo) & 255);
        }
        d = e - (n - 1);
        im.x_out[i] = xx;
        im.d_out[i] = d;
    }
    im.x_out[im.k] = xx + d;
}

// Band 0: fold this tile's best (value, x, d) key into the image's and, on
// the image's last band-0 tile, read the polyline back.
template <typename Acc, typename Hook>
__device__ void finish_band0(unsigned long long best, const ImgDesc &im, const LaunchArgs &args,
                             Hook hook) {
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = best > other ? best : other;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(im.best, best);
    csync();
    if (threadIdx.x == 0) {
        hook();
        __threadfence();
        int prev = atomicAdd(im.done, 1);
        if (prev == im.tiles - 1) readback<Acc>(im, args);
    }
}

__device__ __forceinline__ unsigned long long argmax_key(uint32_t ordv, int x, int eidx) {
    return ((unsigned long long)ordv << 32) | (0xffffffffu - (unsigned)(x * 512 + eidx));
}

// Waits for the three band+1 tiles whose window maxima a tile of `band` reads.
// `after` runs on thread 0 once the flags are seen (or the wait gave up).

// Lanes 0..2 of warp 0 poll the three flags at the same time (a flag already
// seen set by peek_dep is not read again: the fence that follows makes that
// read an acquisition); the warp barrier passes the acquisitions on to lane 0
// and, through the CTA barrier, to every thread.
template <typename After>
__device__ void wait_deps(const ImgDesc &im, int band, int tile, const LaunchArgs &args,
                          After after, int seen = 0) {
    if (band >= im.k - 1) return;
    if (threadIdx.x < 32) {
        const int c = tile - 1 + (int)threadIdx.x;
        bool ok = true;
        if (threadIdx.x < 3 && c >= 0 && c < im.tiles) {
            if (!seen)
                ok = wait_flag(im.flags + (size_t)(band + 1) * im.tiles + c, args.ctl,
                               args.wait_cycles);
            fence_acq_rel_gpu();
        }
        __syncwarp();
        ok = __all_sync(0xffffffffu, ok);
        if (threadIdx.x == 0) {
            if (!ok) atomicExch(&args.ctl->status, FHTDP_ETIMEOUT);
            after();
        }
    }
    csync();
}
__device__ void wait_deps(const ImgDesc &im, int band, int tile, const LaunchArgs &args) {
    wait_deps(im, band, tile, args, [] {});
}

// `before` runs on thread 0 after the CTA barrier, before the flag.
// Every warp fences its own M and bp stores as soon as it is done, so that
// the release by thread 0 after the CTA barrier has little left to wait for.
template <typename Before>
__device__ void publish(const ImgDesc &im, int band, int tile, const LaunchArgs &args,
                        Before before) {
    fence_acq_rel_gpu();
    csync();
    if (threadIdx.x == 0) before();
    const ImgDesc &first = args.many ? args.many[0] : args.one;
    if (band == args.skip_band && tile == args.skip_tile && im.flags == first.flags) return;
    if (threadIdx.x == 0) st_release(im.flags + (size_t)band * im.tiles + tile, 1);
}
__device__ void publish(const ImgDesc &im, int band, int tile, const LaunchArgs &args) {
    publish(im, band, tile, args, [] {});
}

// Stores M_b(x, c) (skewed so that the consumer reads M(x + d, d) as row d,
// column x) and its argmax byte.
template <typename Acc, typename Key>
__device__ __forceinline__ void store_window(const ImgDesc &im, Acc *mnext, int band, int x,
                                             int c, Key mk) {
    using KO = KeyOps<Acc, Key>;
    const int n = im.n;
    const bool dead = mk == KO::dead();
    mnext[(size_t)(c + n - 1) * im.mpitch + kMOff + x - c] = dead ? Dead<Acc>::value()
                                                                  : KO::value(mk);
    im.bp[bp_byte(im, band, c + n - 1, x)] = (uint8_t)(dead ? 0 : KO::index(mk));
}

// Staged uint8 strip of a tile of T columns: columns [x0 - off, x0 + T + off)
// in boxes of 128 columns x n rows.
__host__ __device__ inline int strip_off(int n) { return (n + 15) & ~15; }
__host__ __device__ inline int strip_boxes(int n, int T) {
    return (T + 2 * strip_off(n) + 127) / 128;
}
// One thread: the strip of n image rows from row y0 for (tile, T) through TMA
// into `st` (the Hc region, free until the compaction), zero-filled outside
// the image.
__device__ inline void issue_strip(const CUtensorMap *map, int n, int y0, int tile, int T,
                                   void *st, Pipe &pipe) {
    const int xs = tile * T - strip_off(n), nb = strip_boxes(n, T);
    fence_proxy_async_smem();
    mbar_expect_tx(pipe.bar, (uint32_t)(nb * n * 128));
    for (int b = 0; b < nb; ++b)
        tma_load_2d((uint8_t *)st + (size_t)b * n * 128, map, xs + 128 * b, y0, pipe.bar);
}

// Largest band height a uint8 work item of T = 128 or 256 columns handles
// (its shared-memory regions must fit one CTA).
template <int T>
__host__ __device__ constexpr int max_band() { return T >= 256 ? 64 : 128; }

// ---------------------------------------------------------------------------
// uint8 images.  Shared memory: region A holds the FHT strip F, later V in
// natural displacement order with kPad dead rows on both sides; region Hc
// holds the compact packed Hough words, later the generic window's S.
template <typename Key, bool kMulti>
struct U8Path {
    using Acc = int32_t;
    // The tile width of an item: im.tw in the kernel for batches with both
    // widths, the constant kTile otherwise (every index folds at compile time).
    __device__ static int tw(const ImgDesc &im) { return kMulti ? im.tw : kTile; }
    using KO = KeyOps<int32_t, Key>;
    static constexpr int kRounds = sizeof(Key) == 4 ? 2 : 4;

    // Tiles are T = 128 or 256 columns (im.tw).  Strip rows hold T + n + 15
    // loaded words; the merges read up to T + n + 4.
    __host__ __device__ static int fpitch(int n, int T) { return (T + n + 16 + 3) & ~3; }
    __host__ __device__ static int frows(int n) { return n < 2 ? 2 : n; }
    // V (and the M tile under it) is kept in blocks of 128 columns, each
    // with the 2n-1 displacement rows and kPad dead rows on both sides, so
    // that the window's column stride is a compile-time constant for every
    // tile width: V(row, u) at vblock(n) * (u / 128) + row * 128 + u % 128.
    __host__ __device__ static int vblock(int n) { return (2 * n - 1 + 2 * kPad) * kTile; }
    template <int T>
    __device__ static int vat(int n, int row, int u) {
        if constexpr (T == kTile) return row * kTile + u;
        return (u >> 7) * vblock(n) + row * kTile + (u & (kTile - 1));
    }
    __host__ __device__ static size_t a_bytes(int n, int T) {
        size_t f = (size_t)frows(n) * fpitch(n, T) * 4;
        size_t v = (size_t)vblock(n) * (T / kTile) * 4;
        return ((f > v ? f : v) + 127) / 128 * 128;   // TMA destinations are 128-byte aligned
    }
    __host__ __device__ static size_t hc_bytes(int n, int T) {
        size_t hc = (size_t)n * T * 4;
        size_t s = (size_t)((2 * n - 1 + kRounds - 1) / kRounds) * T * sizeof(Key);
        return hc > s ? hc : s;
    }
    __host__ __device__ static size_t hc_offset();
    // Short bands: the V rows of a tile and the FHT's region F side by side
    // in region A (F after V), so that the M tile can land in the V rows
    // while the FHT runs.
    __host__ __device__ static size_t v_bytes(int n, int T) {
        return ((size_t)vblock(n) * (T / kTile) * 4 + 127) / 128 * 128;
    }
    __host__ __device__ static bool early_m(int n, int T) {
        return v_bytes(n, T) + (size_t)frows(n) * fpitch(n, T) * 4 <= hc_offset();
    }

    // Four pixels [c, c+4) of a row as one little-endian word, zero outside
    // [0, w).  c is a multiple of 4; `aligned` says rows start on 4 bytes.
    __device__ static uint32_t load4(const uint8_t *row, int c, int w, bool aligned) {
        if (aligned && c >= 0 && c + 4 <= w) return __ldg((const uint32_t *)(row + c));
        uint32_t v = 0;
        for (int j = 0; j < 4; ++j) v |= pix_u8(row, c + j, w) << (8 * j);
        return v;
    }

    // Sixteen pixels [c, c+16) of a row, zero outside [0, w); c is a multiple
    // of 16; `aligned` says rows start on 16 bytes.
    __device__ static uint4 load16(const uint8_t *row, int c, int w, bool aligned) {
        if (aligned && c >= 0 && c + 16 <= w) return __ldg((const uint4 *)(row + c));
        uint4 v;
        v.x = load4(row, c, w, false);
        v.y = load4(row, c + 4, w, false);
        v.z = load4(row, c + 8, w, false);
        v.w = load4(row, c + 12, w, false);
        return v;
    }

    // The packed strip, word u of row y = pixel (y, x0 + u) | pixel
    // (y, x0 + T - 1 - u) << 16 (bands of 1 or 2 rows).
    __device__ static void load_strip(uint32_t *F, int pitch, const ImgDesc &im, int band, int x0) {
        const int n = im.n, T = tw(im);
        const int G = (T + n - 1 + 15) / 16;   // groups of 16 strip columns per row
        const uint8_t *base = (const uint8_t *)im.img + (size_t)band * n * im.pitch;
        const bool aligned = ((uintptr_t)im.img % 16 == 0) && (im.pitch % 16 == 0);
        // Word u of strip row y = pixel (y, x0 + u) | pixel (y, x0 + T - 1 - u) << 16:
        // the 16 words [u0, u0+16) take bytes 0..15 of the pixels at x0 + u0 and
        // bytes 15..0 of the pixels at x0 + T - 16 - u0.
#pragma unroll 4
        for (int idx = threadIdx.x; idx < n * G; idx += kThreads) {
            const int y = idx / G, u0 = 16 * (idx - y * G);
            const uint8_t *row = base + (size_t)y * im.pitch;
            const uint4 lo = load16(row, x0 + u0, im.w, aligned);
            const uint4 hi = load16(row, x0 + T - 16 - u0, im.w, aligned);
            const uint32_t los[4] = {lo.x, lo.y, lo.z, lo.w};
            const uint32_t his[4] = {hi.w, hi.z, hi.y, hi.x};
            uint32_t *dst = &F[(size_t)y * pitch + u0];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                uint4 out;
                out.x = __byte_perm(los[g], his[g], 0x0700) & 0x00ff00ffu;
                out.y = __byte_perm(los[g], his[g], 0x0601) & 0x00ff00ffu;
                out.z = __byte_perm(los[g], his[g], 0x0502) & 0x00ff00ffu;
                out.w = __byte_perm(los[g], his[g], 0x0403) & 0x00ff00ffu;
                *(uint4 *)&dst[4 * g] = out;
            }
        }
        csync();
    }

    // Eight pixels [c, c+8) of a row, zero outside [0, w); c is a multiple of
    // 8; `aligned` says rows start on 8 bytes.
    __device__ static uint2 load8(const uint8_t *row, int c, int w, bool aligned) {
        if (aligned && c >= 0 && c + 8 <= w) return __ldg((const uint2 *)(row + c));
        return make_uint2(load4(row, c, w, false), load4(row, c + 4, w, false));
    }

    // Pixels of the band straight from global memory.
    struct GlobalPixels {
        const uint8_t *base;
        long long pitch;
        int w;
        bool aligned;
        __device__ uint2 load8(int row, int X) const {
            return U8Path::load8(base + (size_t)row * pitch, X, w, aligned);
        }
        __device__ uint32_t byte(int row, int X) const {
            return pix_u8(base + (size_t)row * pitch, X, w);
        }
    };
    // Pixels of the band from the strip staged by TMA: box b holds the strip
    // columns [xs + 128b, xs + 128b + 128) of the n band rows, 128 bytes per
    // row; columns outside the image were filled with zeros.  Reads outside
    // the staged columns (they only feed columns past the valid width) are
    // clamped into it.
    struct StagedPixels {
        const uint8_t *st;
        int n, xs, last;   // last = staged bytes per row - 8
        __device__ int clamp(int sc) const { return sc < 0 ? 0 : (sc > last ? last : sc); }
        __device__ uint2 load8(int row, int X) const {
            const int sc = clamp(X - xs);
            return *(const uint2 *)(st + (size_t)(sc >> 7) * n * 128 + row * 128 + (sc & 127));
        }
        __device__ uint32_t byte(int row, int X) const {
            const int sc = clamp(X - xs);
            return st[(size_t)(sc >> 7) * n * 128 + row * 128 + (sc & 127)];
        }
        // 4 bytes at a 4-aligned column inside the staged range (a word
        // never straddles two boxes).
        __device__ uint32_t word(int row, int X) const {
            const int sc = X - xs;
            return *(const uint32_t *)(st + (size_t)(sc >> 7) * n * 128 + row * 128 + (sc & 127));
        }
    };

    // Packed words of N consecutive columns of band row y: word j holds the
    // pixel of column Xp + j (low half) and that of column Xm + 11 - j (high
    // half, the mirrored "-" direction), Xp and Xm 4-aligned, N <= 12.
    template <int N>
    __device__ static void row_words(const StagedPixels &src, int y, int Xp, int Xm,
                                     uint32_t (&P)[N]) {
        constexpr int NW = (N + 3) / 4;
        uint32_t pw[NW], mw[NW];
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            pw[k] = src.word(y, Xp + 4 * k);
            mw[k] = src.word(y, Xm + 4 * (2 - k));
        }
#pragma unroll
        for (int j = 0; j < N; ++j)
            P[j] = __byte_perm(pw[j / 4], mw[j / 4], (j & 3) | ((7 - (j & 3)) << 8)) & 0x00ff00ffu;
    }

    // One level-1 + level-2 step in registers on four rows r0..r0+3 of a
    // sub-band: out[s][u] (s < 4, u < W) from pixel rows of W, W+1, W+2, W+3
    // columns.
    template <int W>
    __device__ static void levels12(const StagedPixels &src, int y0, int Xp, int Xm,
                                    uint32_t (&out)[4][W]) {
        uint32_t A[2][W], Bq[2][W + 2];
        {
            uint32_t p0[W], p1[W + 1];
            row_words(src, y0, Xp, Xm, p0);
            row_words(src, y0 + 1, Xp, Xm, p1);
#pragma unroll
            for (int u = 0; u < W; ++u) {
                A[0][u] = p0[u] + p1[u];
                A[1][u] = p0[u] + p1[u + 1];
            }
        }
        {
            uint32_t p2[W + 2], p3[W + 3];
            row_words(src, y0 + 2, Xp, Xm, p2);
            row_words(src, y0 + 3, Xp, Xm, p3);
#pragma unroll
            for (int u = 0; u < W + 2; ++u) {
                Bq[0][u] = p2[u] + p3[u];
                Bq[1][u] = p2[u] + p3[u + 1];
            }
        }
        // shift s: A_{s>>1}(u) + B_{s>>1}(u + ceil(s/2))
#pragma unroll
        for (int u = 0; u < W; ++u) {
            out[0][u] = A[0][u] + Bq[0][u];
            out[1][u] = A[0][u] + Bq[0][u + 1];
            out[2][u] = A[1][u] + Bq[1][u + 1];
            out[3][u] = A[1][u] + Bq[1][u + 2];
        }
    }

    // Levels 1-3 in registers, straight from the staged pixels (n >= 8): a
    // thread takes an 8-row sub-band g and the 4 columns [4c, 4c+4) of the
    // level-3 width; its top four rows are needed at 4..7 columns, the bottom
    // four at 8..11.  Shift s of the sub-band goes to row 8g + brev3(s).
    __device__ static void fht_regs8(uint32_t *F, int pitch, int n, int T,
                                     const StagedPixels &src, int x0) {
        const int C4 = (T + n - 8 + 3) / 4;
        const int tasks = (n / 8) * C4;
        for (int t = threadIdx.x; t < tasks; t += kThreads) {
            const int g = t / C4, c = t - g * C4;
            const int Xp = x0 + 4 * c, Xm = x0 + T - 12 - 4 * c;
            uint32_t B2[4][8], T2[4][4];
            levels12<8>(src, 8 * g + 4, Xp, Xm, B2);
            levels12<4>(src, 8 * g, Xp, Xm, T2);
            uint32_t *row0 = F + (size_t)(8 * g) * pitch + 4 * c;
            // shift s: T2_{s>>1}(u) + B2_{s>>1}(u + ceil(s/2)), row brev3(s)
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const int h = s >> 1, o = (s + 1) >> 1;
                const int r = ((s & 1) << 2) | (s & 2) | ((s >> 2) & 1);
                *(uint4 *)&row0[(size_t)r * pitch] =
                    make_uint4(T2[h][0] + B2[h][o + 0], T2[h][1] + B2[h][o + 1],
                               T2[h][2] + B2[h][o + 2], T2[h][3] + B2[h][o + 3]);
            }
        }
        csync();
    }

    // Levels 1 and 2 in registers, straight from the pixels: a thread takes 4
    // band rows (a 4-row sub-band g) and 8 strip columns [8c, 8c+8) plus the 3
    // columns after them (from the next lane, which holds chunk c+1), and
    // stores the 4 shifts of the sub-band to rows 4g + brev2(s).
    template <typename Src>
    __device__ static void fht_regs(uint32_t *F, int pitch, int n, int T, const Src &src,
                                    int x0) {
        const int C8 = (T + n - 4 + 7) / 8;   // chunks covering the level-2 width
        const int tasks = (n / 4) * C8;
        const int lane = threadIdx.x & 31;
        for (int t0 = 0; t0 < tasks; t0 += kThreads) {   // uniform: every lane shuffles
            const int t = t0 + threadIdx.x;
            const bool live = t < tasks;
            const int g = live ? t / C8 : 0, c = live ? t - g * C8 : 0;
            uint32_t P[4][11];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int y = 4 * g + r;
                const uint2 lo = live ? src.load8(y, x0 + 8 * c) : make_uint2(0, 0);
                const uint2 hi = live ? src.load8(y, x0 + T - 8 - 8 * c) : make_uint2(0, 0);
                const uint32_t los[2] = {lo.x, lo.y}, his[2] = {hi.y, hi.x};
#pragma unroll
                for (int gg = 0; gg < 2; ++gg) {
                    P[r][4 * gg + 0] = __byte_perm(los[gg], his[gg], 0x0700) & 0x00ff00ffu;
                    P[r][4 * gg + 1] = __byte_perm(los[gg], his[gg], 0x0601) & 0x00ff00ffu;
                    P[r][4 * gg + 2] = __byte_perm(los[gg], his[gg], 0x0502) & 0x00ff00ffu;
                    P[r][4 * gg + 3] = __byte_perm(los[gg], his[gg], 0x0403) & 0x00ff00ffu;
                }
#pragma unroll
                for (int j = 0; j < 3; ++j) P[r][8 + j] = __shfl_down_sync(0xffffffffu, P[r][j], 1);
                // The next chunk of this sub-band is in the next warp: read it.
                if (live && lane == 31 && c + 1 < C8)
                    for (int j = 0; j < 3; ++j) {
                        const int u = 8 * c + 8 + j;
                        P[r][8 + j] = src.byte(y, x0 + u) | (src.byte(y, x0 + T - 1 - u) << 16);
                    }
            }
            // Level 1: rows (0,1) -> A_s', rows (2,3) -> B_s', s' in {0,1}.
            uint32_t A0[8], A1[8], B0[10], B1[10];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                A0[u] = P[0][u] + P[1][u];
                A1[u] = P[0][u] + P[1][u + 1];
            }
#pragma unroll
            for (int v = 0; v < 10; ++v) {
                B0[v] = P[2][v] + P[3][v];
                B1[v] = P[2][v] + P[3][v + 1];
            }
            if (live) {
                // Level 2: shift s -> A_{s>>1}(u) + B_{s>>1}(u + ceil(s/2)).
                uint32_t *row0 = F + (size_t)(4 * g) * pitch + 8 * c;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int u = 4 * h;
                    *(uint4 *)&row0[u] = make_uint4(A0[u] + B0[u], A0[u + 1] + B0[u + 1],
                                                    A0[u + 2] + B0[u + 2], A0[u + 3] + B0[u + 3]);
                    *(uint4 *)&row0[2 * pitch + u] =
                        make_uint4(A0[u] + B0[u + 1], A0[u + 1] + B0[u + 2],
                                   A0[u + 2] + B0[u + 3], A0[u + 3] + B0[u + 4]);
                    *(uint4 *)&row0[pitch + u] =
                        make_uint4(A1[u] + B1[u + 1], A1[u + 1] + B1[u + 2],
                                   A1[u + 2] + B1[u + 3], A1[u + 3] + B1[u + 4]);
                    *(uint4 *)&row0[3 * pitch + u] =
                        make_uint4(A1[u] + B1[u + 2], A1[u + 1] + B1[u + 3],
                                   A1[u + 2] + B1[u + 4], A1[u + 3] + B1[u + 5]);
                }
            }
        }
        csync();
    }

    __host__ __device__ static bool strip_by_tma(const ImgDesc &im) {
        return im.use_tma && im.n >= 4;
    }

    // Returns false if the strip copy did not complete in time.
    // n x T: the strip's rows and columns (a 128-row half of a 256-row band
    // for half-band items, whose strip always comes through TMA).
    __device__ static bool fht(uint32_t *F, uint32_t *Hc, const ImgDesc &im, int band, int x0,
                               Pipe &pipe, bool prefetched, const LaunchArgs &args, int n,
                               int log2n, int T) {
        const int pitch = fpitch(n, T);
        bool compact;
        if (strip_by_tma(im)) {
            const int xs = x0 - strip_off(n), nb = strip_boxes(n, T);
            uint8_t *st = (uint8_t *)Hc;
            if (threadIdx.x == 0 && !prefetched)
                issue_strip(&im.tmap, n, band * n, x0 / T, T, st, pipe);
            const bool ok = mbar_wait(pipe.bar, pipe.phase, args.wait_cycles);
            if (!ok) {
                // The copy may still be in flight: give it a long (bounded)
                // last chance to land before Hc is written again.
                if (threadIdx.x == 0) atomicExch(&args.ctl->status, FHTDP_ETIMEOUT);
                mbar_wait(pipe.bar, pipe.phase, kDrainCycles);
                pipe.phase ^= 1u;
                return false;
            }
            pipe.phase ^= 1u;
            const StagedPixels src{st, n, xs, nb * 128 - 8};
            if (n >= 8 && im.depth == 3) {
                fht_regs8(F, pitch, n, T, src, x0);
                compact = !fht_merge<uint32_t>(F, pitch, n, log2n, T, 4, Hc);
            } else {
                fht_regs(F, pitch, n, T, src, x0);
                compact = !fht_merge<uint32_t>(F, pitch, n, log2n, T, 3, Hc);
            }
        } else if (n >= 4) {
            const GlobalPixels src{(const uint8_t *)im.img + (size_t)band * n * im.pitch,
                                   im.pitch, im.w,
                                   ((uintptr_t)im.img % 8 == 0) && (im.pitch % 8 == 0)};
            fht_regs(F, pitch, n, T, src, x0);
            compact = !fht_merge<uint32_t>(F, pitch, n, log2n, T, 3, Hc);
        } else {
            load_strip(F, pitch, im, band, x0);
            compact = log2n == 0;
            fht_levels<uint32_t>(F, pitch, n, log2n, T, 1, Hc);
        }
        // The last level wrote Hc[s][u] = packed Hough word of shift s at tile
        // column u; where the FHT had no merge level (n = 1, or n = 4 done in
        // registers) the words are copied from their bit-reversed rows.
        if (compact) {
            for (int idx = threadIdx.x; idx < n * (T / 4); idx += kThreads) {
                const int s = idx / (T / 4), u0 = 4 * (idx - s * (T / 4));
                *(uint4 *)&Hc[s * T + u0] =
                    *(const uint4 *)&F[(size_t)brev(s, log2n) * pitch + u0];
            }
            csync();
        }
        return true;
    }

    // V rows: V(e) of tile column u at Vn[(e + n - 1 + kPad) * T + u].
    // M buffer words.  With 32-bit keys a window maximum is kept as its key
    // with the index bits cleared, M' = value << 9 (negative when dead), so
    // that a V key is M' + (H << 9 | index); 64-bit keys keep the value.
    __device__ static int32_t mstore(Key mk) {
        if constexpr (sizeof(Key) == 4) return mk & ~511;
        else return mk < 0 ? Dead<int32_t>::value() : KO::value(mk);
    }
    __device__ static int32_t mval(int32_t w) {
        if constexpr (sizeof(Key) == 4) return w >> 9;
        else return w;
    }
    // The kPad dead rows above and below the V rows.
    template <int T>
    __device__ static void dead_pad(int32_t *Vn, int n) {
        const int D = 2 * n - 1;
        const int32_t dead = Dead<int32_t>::value();
        for (int idx = threadIdx.x; idx < 2 * kPad * (T / 4); idx += kThreads) {
            const int r = idx / (T / 4), u0 = 4 * (idx % (T / 4));
            const int row = r < kPad ? r : r + D;
            *(int4 *)&Vn[vat<T>(n, row, u0)] = make_int4(dead, dead, dead, dead);
        }
    }
    // V keys of an interior tile, in place over the M' tile copied by TMA
    // (none in the last band): V key(c) = M'(c) + (H(c) << 9 | 511 - (c + n - 1)).
    // A dead M' (negative) gives a negative key.
    template <int T>
    __device__ static void form_v_interior(int32_t *Vn, const uint32_t *Hc, int n, bool last) {
        const int kc = 512 - n;   // 511 - (c + n - 1) = kc - c
        for (int idx = threadIdx.x; idx < n * (T / 4); idx += kThreads) {
            const int s = idx / (T / 4), u0 = 4 * (idx % (T / 4));
            const uint4 hw = *(const uint4 *)&Hc[s * T + u0];
            int4 *pp = (int4 *)&Vn[vat<T>(n, s + n - 1 + kPad, u0)];
            int4 *pm = (int4 *)&Vn[vat<T>(n, n - 1 - s + kPad, T - 4 - u0)];
            int4 mp = make_int4(0, 0, 0, 0), mm = mp;
            if (!last) {
                mp = *pp;
                if (s > 0) mm = *pm;
            }
            const int kp = kc - s, km = kc + s;
            *pp = make_int4(mp.x + (int)(hw.x & 0xffffu) * 512 + kp,
                            mp.y + (int)(hw.y & 0xffffu) * 512 + kp,
                            mp.z + (int)(hw.z & 0xffffu) * 512 + kp,
                            mp.w + (int)(hw.w & 0xffffu) * 512 + kp);
            // "-" half of word j is column T - 1 - u0 - j, at pm lane 3 - j.
            if (s > 0)
                *pm = make_int4(mm.x + (int)(hw.w >> 16) * 512 + km,
                                mm.y + (int)(hw.z >> 16) * 512 + km,
                                mm.z + (int)(hw.y >> 16) * 512 + km,
                                mm.w + (int)(hw.x >> 16) * 512 + km);
        }
    }
    // With msmem the M tile was copied by TMA into the V rows (row e of M at
    // V row e + kPad), and V is formed in place; otherwise M is read from L2.
    template <int T>
    __device__ static unsigned long long form_v(int32_t *Vn, const uint32_t *Hc,
                                                const ImgDesc &im, int band, int x0,
                                                const int32_t *mprev, bool msmem) {
        const int n = im.n;
        const bool last = band == im.k - 1;
        const Acc dead = Dead<Acc>::value();
        int wlo, whi;
        band_window(im, band, &wlo, &whi);
        unsigned long long best = 0;
        // The M loads of a batch of iterations are issued before any of its
        // shared stores, so their L2 round trips overlap.
        // At most 128 x 128 / 4 or 64 x 256 / 4 tasks: 8 per thread.
        constexpr int kIt = kMaxBandFused * (kTile / 4) / kThreads;
        constexpr int kLB = 4;
        const int tasks = n * (T / 4);
#pragma unroll 1
        for (int b0 = 0; b0 < kIt; b0 += kLB) {
        if (threadIdx.x + b0 * kThreads >= tasks) break;
        int4 mpa[kLB], mma[kLB];
#pragma unroll
        for (int i = 0; i < kLB; ++i) {
            const int idx = threadIdx.x + (b0 + i) * kThreads;
            const int s = idx / (T / 4), u0 = 4 * (idx % (T / 4));
            mpa[i] = make_int4(0, 0, 0, 0);
            mma[i] = mpa[i];
            if (!last && idx < tasks) {
                if (msmem) {
                    mpa[i] = *(const int4 *)&Vn[vat<T>(n, s + n - 1 + kPad, u0)];
                    if (s > 0)
                        mma[i] = *(const int4 *)&Vn[vat<T>(n, n - 1 - s + kPad, T - 4 - u0)];
                } else {
                    mpa[i] = __ldcg((const int4 *)(mprev + (size_t)(s + n - 1) * im.mpitch +
                                                   kMOff + x0 + u0));
                    if (s > 0)
                        mma[i] = __ldcg((const int4 *)(mprev + (size_t)(n - 1 - s) * im.mpitch +
                                                       kMOff + x0 + T - 4 - u0));
                }
            }
        }
#pragma unroll
        for (int it = 0; it < kLB; ++it) {
            const int idx = threadIdx.x + (b0 + it) * kThreads;
            if (idx >= tasks) break;
            const int s = idx / (T / 4), u0 = 4 * (idx % (T / 4));
            const uint4 hw = *(const uint4 *)&Hc[s * T + u0];
            const uint32_t hws[4] = {hw.x, hw.y, hw.z, hw.w};
            // "+" half: column x0 + u0 + j, displacement +s.
            const int xp = x0 + u0;
            const int4 mp = mpa[it], mm = mma[it];
            const int mps[4] = {mp.x, mp.y, mp.z, mp.w};
            const int mms[4] = {mm.x, mm.y, mm.z, mm.w};   // column x0 + T - 4 - u0 + t
            int vp[4], vm[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int x = xp + j;
                const bool ok = x < im.w && x + s < im.w && s >= wlo && s <= whi;
                // A window maximum below zero marks a dead continuation
                // (uint8 sums are never negative).
                const int m = mval(mps[j]);
                vp[j] = !ok ? dead : last ? (int)(hws[j] & 0xffffu)
                                          : (m < 0 ? dead : (int)(hws[j] & 0xffffu) + m);
                // "-" half of word j: column x0 + T - 1 - u0 - j, displacement -s.
                const int xm = x0 + T - 1 - u0 - j;
                const bool okm = s > 0 && xm < im.w && xm - s >= 0 && -s >= wlo && -s <= whi;
                const int mmv = mval(mms[3 - j]);
                vm[j] = !okm ? dead : last ? (int)(hws[j] >> 16)
                                           : (mmv < 0 ? dead : (int)(hws[j] >> 16) + mmv);
            }
            if (band == 0) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (vp[j] != dead) {
                        const unsigned long long k = argmax_key(ord32(vp[j]), xp + j, s + n - 1);
                        best = best > k ? best : k;
                    }
                    if (vm[j] != dead) {
                        const unsigned long long k =
                            argmax_key(ord32(vm[j]), x0 + T - 1 - u0 - j, n - 1 - s);
                        best = best > k ? best : k;
                    }
                }
            } else {
                if constexpr (sizeof(Key) == 4) {
                    // Store window keys: value << 9 | (511 - (e + n - 1)); dead
                    // stays INT32_MIN.
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        vp[j] = vp[j] == dead ? dead : KO::make(vp[j], s + n - 1);
                        vm[j] = vm[j] == dead ? dead : KO::make(vm[j], n - 1 - s);
                    }
                }
                *(int4 *)&Vn[vat<T>(n, s + n - 1 + kPad, u0)] =
                    make_int4(vp[0], vp[1], vp[2], vp[3]);
                if (s > 0)
                    *(int4 *)&Vn[vat<T>(n, n - 1 - s + kPad, T - 4 - u0)] =
                        make_int4(vm[3], vm[2], vm[1], vm[0]);
            }
        }
        }
        return best;
    }

    // Subproblems 2-3: the states of the point's band whose vertex on the
    // point's border is not mask_x become dead (their link's start x, or for
    // the image's bottom border its end x + e), in V once it is formed: the
    // same restriction as the standalone point mask.
    template <int T>
    __device__ static void mask_point(int32_t *Vn, const ImgDesc &im, int x0) {
        const int n = im.n, D = 2 * n - 1;
        for (int idx = threadIdx.x; idx < D * T; idx += kThreads) {
            const int ei = idx / T, u = idx - ei * T;
            const int x = x0 + u;
            if ((im.mask_end ? x + ei - (n - 1) : x) != im.mask_x)
                Vn[vat<T>(n, ei + kPad, u)] = INT32_MIN;   // dead in keys and in values
        }
    }

    // Thread 0: takes the next work item and, when its strip can go to Hc
    // now (Hc is not needed any more by this item), issues the strip copy.
    // The compute warps' part of a work item.  The control warp issued the
    // item's strip copy; after the FHT it copies the M tile (or, where there
    // is none, just signals that the producers' flags were seen) on the M
    // barrier.  A wait that gives up sets ETIMEOUT and the item carries on,
    // so that every signal to the control warp is still given.
    // half >= 0: a half-band FHT item of a 256-row band (its FHT only).
    __device__ static void process(const ImgDesc &im, int band, int tile, unsigned char *smem,
                                   const LaunchArgs &args, Pipe &pipe, bool prefetched,
                                   int half) {
        const bool hitem = kMulti && half >= 0;
        const int n = hitem ? 128 : im.n, T = hitem ? kTile : tw(im), D = 2 * n - 1;
        const int x0 = tile * T;
        // the FHT's region; after V when both fit (the M tile may then come
        // during the FHT)
        uint32_t *F = (uint32_t *)(smem + (!hitem && early_m(n, T) ? v_bytes(n, T) : 0));
        int32_t *Vn = (int32_t *)smem;
        uint32_t *Hc = (uint32_t *)(smem + hc_offset());
        fht(F, Hc, im, band, x0, pipe, prefetched, args, n, hitem ? 7 : im.log2n, T);
        nb_arrive(kBarFhtDone, kCtlSync);   // F is free for the M tile (if it overlaps V)
        if (hitem) {
            store_half(im, band, half, x0, Hc);
            nb_arrive(kBarHcFree, kCtlSync);
            nb_arrive(kBarWinDone, kCtlSync);
            return;
        }
        const bool msmem = im.use_mtma && band < im.k - 1;
        if (band != 0) {
            if (T == kTile) dead_pad<kTile>(Vn, n);
            else dead_pad<2 * kTile>(Vn, n);
        }
        if (!mbar_wait(pipe.mbar, pipe.mphase, args.wait_cycles)) {
            // As for the strip: the M copy lands in the V rows, so let it
            // finish (bounded) before V is formed there.
            if (threadIdx.x == 0) atomicExch(&args.ctl->status, FHTDP_ETIMEOUT);
            mbar_wait(pipe.mbar, pipe.mphase, kDrainCycles);
        }
        pipe.mphase ^= 1u;
        const Acc *mprev = (const Acc *)im.mbuf[(band + 1) & 1];
        Acc *mnext = (Acc *)im.mbuf[band & 1];
        const bool fast = sizeof(Key) == 4 && im.B <= kFastB;
        // Interior tiles (every x - s and x + s of the tile inside the image)
        // of a band without windows need no masks.
        const bool interior = sizeof(Key) == 4 && band != 0 && !im.win &&
                              (msmem || band == im.k - 1) &&
                              x0 >= n - 1 && x0 + T + n - 2 < im.w;
        unsigned long long best = 0;
        if (T == kTile) {
            if (interior) form_v_interior<kTile>(Vn, Hc, n, band == im.k - 1);
            else best = form_v<kTile>(Vn, Hc, im, band, x0, mprev, msmem);
        } else {
            if (interior) form_v_interior<2 * kTile>(Vn, Hc, n, band == im.k - 1);
            else best = form_v<2 * kTile>(Vn, Hc, im, band, x0, mprev, msmem);
        }
        if (band == 0) {
            // The tile's best key; the control warp counts the tile and reads
            // the polyline back after the image's last one.
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
                best = best > other ? best : other;
            }
            if ((threadIdx.x & 31) == 0 && best) atomicMax(im.best, best);
            nb_arrive(kBarHcFree, kCtlSync);
            nb_arrive(kBarWinDone, kCtlSync);
            return;
        }
        csync();
        if (band + 1 == im.mask1) {   // the through-point band (never band 0)
            if (T == kTile) mask_point<kTile>(Vn, im, x0);
            else mask_point<2 * kTile>(Vn, im, x0);
            csync();
        }
        // Hc is free from here on unless the window reads S from it.
        if (fast) nb_arrive(kBarHcFree, kCtlSync);

        // T / 128 = 1 or 2 column blocks; kQ = 512 / T threads per column.
        const int lt = T == 256 ? 8 : 7, kq = kThreads >> lt;
        const int u = threadIdx.x & (T - 1), qd = threadIdx.x >> lt;
        const int x = x0 + u;
        const int B = im.B;   // already clamped to 2n-2
        const int lo = -(n - 1), hi = n - 1;
        const int32_t *col = Vn + vat<2 * kTile>(n, 0, u);   // row stride kTile
        if constexpr (sizeof(Key) == 4) {
            if (B <= kFastB) {
                // Shared memory holds keys.  V rows [lo - kPad, hi + kPad] exist
                // (dead outside [lo, hi]), and B <= kPad: the register window
                // reads them without bounds checks.
                const int32_t *kcol = col + (n - 1 + kPad) * kTile;
                // M'(x, c) = key & ~511 (negative when dead), bp = its index.
                Acc *mcol = mnext + (size_t)(n - 1) * im.mpitch + kMOff + x;
                const int mstep = im.mpitch - 1;
                // Quarters of the displacement indices e = c + n - 1, cut at
                // multiples of 4 (whole bp words).  Only the consumer band's
                // allowed displacements are needed; a thread starts at the word
                // boundary below them (the extra maxima are never read).
                const int Q = 4 * (((D + 3) / 4 + kq - 1) / kq);
                int clo, chi;
                band_window(im, band - 1, &clo, &chi);
                const int ea = max(qd * Q, (clo + n - 1) & ~3);
                const int e1 = min(min((qd + 1) * Q, D) - 1, chi + n - 1);
                if (ea <= e1 && x < im.w) {
                    const int ca = ea - (n - 1), c1 = e1 - (n - 1);
                    uint32_t *bw = (uint32_t *)im.bp +
                                   ((size_t)band * bp_groups(n) + (ea >> 2)) * im.w + x;
                    int32_t *ma = mcol + (long long)ca * mstep;
                    switch (B) {
                        case 4: window_u8<9>(ca, c1, kcol, ma, mstep, bw, im.w); break;
                        case 8: window_u8<17>(ca, c1, kcol, ma, mstep, bw, im.w); break;
                        case 12: window_u8<25>(ca, c1, kcol, ma, mstep, bw, im.w); break;
                        case 16: window_u8<33>(ca, c1, kcol, ma, mstep, bw, im.w); break;
                        default: {
                            const Key dk = KO::dead();
                            auto vkey = [&](int e) -> Key { return kcol[e * kTile]; };
                            auto emit = [&](int c, Key mk) {
                                mcol[(long long)c * mstep] = mk & ~511;
                                im.bp[bp_byte(im, band, c + n - 1, x)] = (uint8_t)(~mk & 255);
                            };
                            if (B < 4)
                                window_regs<9, false, Key>(ca, c1, B, dk, vkey, emit);
                            else if (B < 8)
                                window_regs<17, false, Key>(ca, c1, B, dk, vkey, emit);
                            else
                                window_regs<33, false, Key>(ca, c1, B, dk, vkey, emit);
                        }
                    }
                }
                nb_arrive(kBarWinDone, kCtlSync);
                return;
            }
        }
        auto emit = [&](int c, Key mk) {
            mnext[(size_t)(c + n - 1) * im.mpitch + kMOff + x - c] = mstore(mk);
            im.bp[bp_byte(im, band, c + n - 1, x)] = (uint8_t)(mk < 0 ? 0 : KO::index(mk));
        };
        {
            auto vkey = [&](int e) -> Key {
                if (e < lo || e > hi) return KO::dead();
                const int v = col[(e + n - 1 + kPad) * kTile];
                if constexpr (sizeof(Key) == 4) return v;   // stored as keys
                return v == Dead<Acc>::value() ? KO::dead() : KO::make(v, e + n - 1);
            };
            Key *S = (Key *)Hc;
            for (int round = 0; round < kRounds; ++round) {
                const int P0 = lo + (round * D) / kRounds;
                const int P1 = lo + ((round + 1) * D) / kRounds - 1;
                const int span = P1 - P0 + 1;
                int clo, chi;
                band_window(im, band - 1, &clo, &chi);
                const int c0 = max(P0 + (qd * span) / kq, clo);
                const int c1 = min(P0 + ((qd + 1) * span) / kq - 1, chi);
                const int srow0 = P0 - B;   // S(e) at row e - srow0
                auto sput = [&](int e, Key v) { S[(size_t)(e - srow0) * T + u] = v; };
                auto sget = [&](int e) { return S[(size_t)(e - srow0) * T + u]; };
                if (c0 <= c1 && x < im.w)
                    window_two_pass<Key>(c0, c1, B, lo - B, lo, hi, KO::dead(), vkey, sput, sget,
                                         emit);
                csync();
            }
        }
        nb_arrive(kBarHcFree, kCtlSync);
        nb_arrive(kBarWinDone, kCtlSync);
    }

    // ---------------------------------------------------------------------
    // 256-row bands.  A link over the band's 256 rows is, by the last level
    // of Sec. 2.1's dyadic recursion, a link of shift s over the top 128 rows
    // followed by one of shift s over the bottom 128 rows, moved by s + r:
    //   H(x, 2s + r)    = Htop+(x, s) + Hbot+(x + s + r, s)
    //   H(x, -(2s + r)) = Htop-(x, s) + Hbot-(x - s - r, s),   s < 128, r in {0, 1}.
    // Half-band items compute the FHT of one 128-row half for 128 columns
    // and store it to h256; the DP items of 64 columns apply that last level
    // while they form V.
    __device__ static uint16_t *h256_row(const ImgDesc &im, int band, int half, int sign,
                                         int s) {
        return im.h256 + ((((size_t)band * 2 + half) * 2 + sign) * 128 + s) * im.hpitch +
               kH256Left;
    }

    // The FHT of one 128-row half of a 256-row band on a tile of 128 columns,
    // from its compact rows in Hc into h256.  Word u of shift s holds the
    // right-moving sum from column x0 + u in its low half and the
    // left-moving sum from column x0 + 127 - u in its high half: 8 words
    // give 8 columns of each sign.
    __device__ static void store_half(const ImgDesc &im, int band, int half, int x0,
                                      const uint32_t *Hc) {
        constexpr int n = 128, T = kTile;
        for (int idx = threadIdx.x; idx < n * (T / 8); idx += kThreads) {
            const int sh = idx >> 4, q = idx & 15;
            const uint4 a = *(const uint4 *)&Hc[sh * T + 8 * q];
            const uint4 b = *(const uint4 *)&Hc[sh * T + 8 * q + 4];
            *(uint4 *)(h256_row(im, band, half, 0, sh) + x0 + 8 * q) =
                make_uint4(__byte_perm(a.x, a.y, 0x5410), __byte_perm(a.z, a.w, 0x5410),
                           __byte_perm(b.x, b.y, 0x5410), __byte_perm(b.z, b.w, 0x5410));
            *(uint4 *)(h256_row(im, band, half, 1, sh) + x0 + T - 8 - 8 * q) =
                make_uint4(__byte_perm(b.w, b.z, 0x7632), __byte_perm(b.y, b.x, 0x7632),
                           __byte_perm(a.w, a.z, 0x7632), __byte_perm(a.y, a.x, 0x7632));
        }
    }

    // The DP of a 64-column tile of a 256-row band: V (Eqs. 3-4) from the two
    // halves' FHTs and the M tile, then the bend-window maxima (two-pass van
    // Herk / Gil-Werman).  V(e) of column u is at Vn[(e + n - 1 + kPad) * 64 + u].
    __device__ static void process_dp256(const ImgDesc &im, int band, int tile,
                                         unsigned char *smem, const LaunchArgs &args,
                                         Pipe &pipe) {
        constexpr int n = 256, T = kTile256, D = 2 * n - 1;
        const int x0 = tile * T;
        int32_t *Vn = (int32_t *)smem;
        nb_arrive(kBarFhtDone, kCtlSync);   // no FHT here: the M tile may come at once
        const bool last = band == im.k - 1;
        const int32_t dead = Dead<int32_t>::value();
        if (band != 0)
            for (int idx = threadIdx.x; idx < 2 * kPad * (T / 4); idx += kThreads) {
                const int r = idx / (T / 4), u0 = 4 * (idx % (T / 4));
                const int row = r < kPad ? r : r + D;
                *(int4 *)&Vn[row * T + u0] = make_int4(dead, dead, dead, dead);
            }
        if (!mbar_wait(pipe.mbar, pipe.mphase, args.wait_cycles)) {
            if (threadIdx.x == 0) atomicExch(&args.ctl->status, FHTDP_ETIMEOUT);
            mbar_wait(pipe.mbar, pipe.mphase, kDrainCycles);
        }
        pipe.mphase ^= 1u;
        // A task: shift s of the halves, one sign, 4 columns; it forms the
        // displacements 2s and 2s + 1 (d = 0 once, with sign 0).  The L2
        // loads of a batch of tasks are issued before any of its work.
        unsigned long long best = 0;
        constexpr int kTasks = 2 * 128 * (T / 4), kLB = 8;
        static_assert(kTasks % (kLB * kThreads) == 0, "whole batches");
#pragma unroll 1
        for (int b0 = 0; b0 < kTasks; b0 += kLB * kThreads) {
            uint2 aw[kLB];
            uint32_t bw[kLB][3];
            int base[kLB];
#pragma unroll
            for (int i = 0; i < kLB; ++i) {
                const int idx = b0 + i * kThreads + threadIdx.x;
                const int q = idx & 15, sh = (idx >> 4) & 127, sign = idx >> 11;
                const int x = x0 + 4 * q;
                aw[i] = __ldcg((const uint2 *)(h256_row(im, band, 0, sign, sh) + x));
                // The bottom half from column base: x + s (right) or x - s - 1 (left).
                base[i] = sign ? x - sh - 1 : x + sh;
                const uint32_t *bp =
                    (const uint32_t *)(h256_row(im, band, 1, sign, sh) + (base[i] & ~1));
                bw[i][0] = __ldcg(bp);
                bw[i][1] = __ldcg(bp + 1);
                bw[i][2] = __ldcg(bp + 2);
            }
#pragma unroll
            for (int i = 0; i < kLB; ++i) {
            const int idx = b0 + i * kThreads + threadIdx.x;
            const int q = idx & 15, sh = (idx >> 4) & 127, sign = idx >> 11;
            const int x = x0 + 4 * q;
            const int fs = (base[i] & 1) * 16;
            const uint32_t p0 = __funnelshift_r(bw[i][0], bw[i][1], fs);
            const uint32_t p1 = __funnelshift_r(bw[i][1], bw[i][2], fs);
            const int av[4] = {(int)(aw[i].x & 0xffffu), (int)(aw[i].x >> 16),
                               (int)(aw[i].y & 0xffffu), (int)(aw[i].y >> 16)};
            const int bv[5] = {(int)(p0 & 0xffffu), (int)(p0 >> 16), (int)(p1 & 0xffffu),
                               (int)(p1 >> 16),
                               (int)(fs ? bw[i][2] >> 16 : bw[i][2] & 0xffffu)};
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int e = 2 * sh + r;
                if (sign && e == 0) continue;
                const int d = sign ? -e : e;
                const int row = d + n - 1 + kPad;
                // right: x + s + r + j = base + r + j; left: x - s - r + j = base + 1 - r + j
                const int bo = sign ? 1 - r : r;
                int4 m4 = make_int4(0, 0, 0, 0);
                if (!last) m4 = *(const int4 *)&Vn[row * T + 4 * q];
                const int ms[4] = {m4.x, m4.y, m4.z, m4.w};
                int v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int xx = x + j;
                    const bool ok = xx < im.w && xx + d >= 0 && xx + d < im.w;
                    const int hv = av[j] + bv[j + bo];
                    const int m = mval(ms[j]);
                    v[j] = !ok ? dead : last ? hv : (m < 0 ? dead : hv + m);
                }
                if (band == 0) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (v[j] != dead) {
                            const unsigned long long k = argmax_key(ord32(v[j]), x + j, d + n - 1);
                            best = best > k ? best : k;
                        }
                } else {
                    if constexpr (sizeof(Key) == 4) {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            v[j] = v[j] == dead ? dead : KO::make(v[j], d + n - 1);
                    }
                    *(int4 *)&Vn[row * T + 4 * q] = make_int4(v[0], v[1], v[2], v[3]);
                }
            }
        }
        }
        if (band == 0) {
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
                best = best > other ? best : other;
            }
            if ((threadIdx.x & 31) == 0 && best) atomicMax(im.best, best);
            nb_arrive(kBarHcFree, kCtlSync);
            nb_arrive(kBarWinDone, kCtlSync);
            return;
        }
        csync();
        // Window maxima.  32-bit keys with 16 <= B <= 32: 16 threads per
        // column, 32 displacements each (window_span32), two columns per
        // thread.  Otherwise 8 threads per column over 64 displacements.
        const int B = im.B;
        const int lo = -(n - 1), hi = n - 1;
        Acc *mnext = (Acc *)im.mbuf[band & 1];
        if (sizeof(Key) == 4 && B >= 16 && B <= 32) {
            const int qd = threadIdx.x >> 5;   // displacements [lo + 32 qd, lo + 32 qd + 31]
            const int c0 = lo + 32 * qd;
            for (int u = threadIdx.x & 31; u < T; u += 32) {
                const int xw = x0 + u;
                if (xw >= im.w) continue;
                const int32_t *col = Vn + (n - 1 + kPad) * T + u;
                auto vkey = [&](int e) -> int32_t {
                    return (e < lo || e > hi) ? INT32_MIN : col[e * T];
                };
                int32_t *mcol = mnext + (size_t)(c0 + n - 1) * im.mpitch + im.moff + xw - c0;
                uint32_t *bw = (uint32_t *)im.bp +
                               ((size_t)band * bp_groups(n) + ((c0 + n - 1) >> 2)) * im.w + xw;
                // the last thread's 32nd displacement (c = n) does not exist
                window_span32(c0, min(32, hi - c0 + 1), B, vkey, mcol, im.mpitch - 1, bw, im.w);
            }
            nb_arrive(kBarHcFree, kCtlSync);
            nb_arrive(kBarWinDone, kCtlSync);
            return;
        }
        const int u = threadIdx.x & (T - 1), qd = threadIdx.x / T;
        const int xw = x0 + u;
        const int32_t *col = Vn + (n - 1 + kPad) * T + u;
        auto vkey = [&](int e) -> Key {
            if (e < lo || e > hi) return KO::dead();
            const int v = col[e * T];
            if constexpr (sizeof(Key) == 4) return v;   // stored as keys
            return v == dead ? KO::dead() : KO::make(v, e + n - 1);
        };
        // The backpointer byte keeps the argmax index modulo 256 (the
        // read-back recovers it from the window, B <= 127).
        auto emit = [&](int c, Key mk) {
            mnext[(size_t)(c + n - 1) * im.mpitch + im.moff + xw - c] = mstore(mk);
            im.bp[bp_byte(im, band, c + n - 1, xw)] = (uint8_t)(mk < 0 ? 0 : KO::index(mk));
        };
        const int c0 = lo + 64 * qd, c1 = min(c0 + 63, hi);
        if (sizeof(Key) == 4 && B < 16) {
            if (xw < im.w) window_reread<17, Key>(c0, c1, B, KO::dead(), vkey, emit);
        } else {
            // Longer windows: the two-pass version with S in shared memory
            // after V (64 rows per thread), a few of the column's threads at a
            // time so that S fits (64 KB).
            constexpr int kGroups = sizeof(Key) == 4 ? 2 : 4, kPer = 8 / kGroups;
            for (int g = 0; g < kGroups; ++g) {
                if (qd / kPer == g && xw < im.w) {
                    Key *S = (Key *)(smem + kDp256SOff) + (size_t)(qd % kPer) * 64 * T;
                    const int srow0 = c0 - B;   // S(e) at row e - srow0
                    auto sput = [&](int e, Key v) { S[(size_t)(e - srow0) * T + u] = v; };
                    auto sget = [&](int e) { return S[(size_t)(e - srow0) * T + u]; };
                    window_two_pass<Key>(c0, c1, B, lo - B, lo, hi, KO::dead(), vkey, sput, sget,
                                         emit);
                }
                csync();
            }
        }
        nb_arrive(kBarHcFree, kCtlSync);
        nb_arrive(kBarWinDone, kCtlSync);
    }
};

// Shared-memory layout common to the uint8 items of every tile width: region
// A from offset 0, Hc at a fixed offset (the largest region A), so that the
// strip of a next item with another band height or tile width can be staged
// in Hc while the current item still uses region A.
template <typename Key>
__host__ __device__ size_t u8_hc_offset() {
    const size_t a = U8Path<Key, true>::a_bytes(max_band<128>(), 128);
    const size_t b = U8Path<Key, true>::a_bytes(max_band<256>(), 256);
    return a > b ? a : b;
}
template <typename Key>
size_t u8_smem_bytes() {
    const size_t a = U8Path<Key, true>::hc_bytes(max_band<128>(), 128);
    const size_t b = U8Path<Key, true>::hc_bytes(max_band<256>(), 256);
    return u8_hc_offset<Key>() + (a > b ? a : b);
}
template <typename Key, bool kMulti>
__host__ __device__ size_t U8Path<Key, kMulti>::hc_offset() { return u8_hc_offset<Key>(); }

// The control warp of the uint8 engine (items of any tile width).
template <typename Key>
struct U8Ctl {
    // An item as the control warp sees it.
    struct Ctrl {
        long long item;
        const ImgDesc *im;
        int band, tile, n, T, kind;
        bool tma;   // its strip goes through TMA
    };
    // Work items of a single image with 256-row bands, in queue order: the
    // half-band FHT items of band k-1, then per band b from k-1 down to 0
    // the half-band items of band b-1 (none for b = 0) and the DP items of b.
    __device__ static void decode256(const ImgDesc &im, long long item, Ctrl &c) {
        const long long hf = 2LL * im.ftiles, L1 = hf + im.tiles;
        if (item < hf) {
            c.band = im.k - 1;
            c.kind = kItemHalf0 + (int)(item / im.ftiles);
            c.tile = (int)(item % im.ftiles);
            return;
        }
        const long long j = item - hf;
        long long lv = j / L1, off = j - lv * L1;
        if (lv >= im.k - 1) {
            lv = im.k - 1;
            off = j - (long long)(im.k - 1) * L1;
        }
        const int b = im.k - 1 - (int)lv;
        if (b > 0 && off < hf) {
            c.band = b - 1;
            c.kind = kItemHalf0 + (int)(off / im.ftiles);
            c.tile = (int)(off % im.ftiles);
        } else {
            c.band = b;
            c.kind = kItemDp256;
            c.tile = (int)(off - (b > 0 ? hf : 0));
        }
    }
    // The first item from `item` on (an index just taken from the queue)
    // whose image is enabled, taking more as needed (lane 0).
    __device__ static long long skip_disabled(const LaunchArgs &args, long long item) {
        for (;;) {
            if (item >= args.items || !args.many) return item;
            const ImgDesc *im = &args.many[args.order[item].image];
            if (!im->enable || __ldcg(im->enable) != 0) return item;
            item = atomicAdd(&args.ctl->queue, 1);
        }
    }
    // The next item of the queue whose image is enabled (lane 0 takes it).
    __device__ static long long take(const LaunchArgs &args) {
        return skip_disabled(args, atomicAdd(&args.ctl->queue, 1));
    }
    __device__ static Ctrl decode(const LaunchArgs &args, long long item) {
        Ctrl c{item, nullptr, 0, 0, 0, 128, kItemBand, false};
        if (item >= args.items) return c;
        if (args.many) {
            const Item it = args.order[item];
            c.im = &args.many[it.image];
            c.band = it.band;
            c.tile = it.tile;
            c.n = it.nflags & 0xffff;
            c.kind = (it.nflags >> 19) & 3;
            c.tma = ((it.nflags >> 16) & 1) && c.n >= 4;
            c.T = 64 << ((it.nflags >> 17) & 3);
        } else {
            c.im = &args.one;
            c.n = args.one.n;
            c.tma = args.one.use_tma && c.n >= 4;
            c.T = args.one.tw;
            if (args.one.kind == 1) {
                decode256(args.one, item, c);
            } else {
                c.band = args.one.k - 1 - (int)(item / args.one.tiles);
                c.tile = (int)(item % args.one.tiles);
            }
        }
        if (c.kind == kItemHalf0 || c.kind == kItemHalf1) {
            c.n = 128;   // the strip of one half
            c.T = kTile;
        } else if (c.kind == kItemDp256) {
            c.tma = false;   // no strip
        }
        return c;
    }
    // Lane 0: the item's strip copy into Hc, and its slot for the compute warps.
    __device__ static void hand_over(const Ctrl &c, WsSlot *slot, void *Hc, Pipe &pipe) {
        if (c.im && c.tma) {
            const int y0 = c.kind == kItemBand ? c.band * c.n
                                               : c.band * 256 + (c.kind - kItemHalf0) * 128;
            issue_strip(&c.im->tmap, c.n, y0, c.tile, c.T, Hc, pipe);
        }
        slot->item = c.item;
        slot->im = c.im;
        slot->band = c.band;
        slot->tile = c.tile;
        slot->T = c.T;
        slot->kind = c.kind;
        slot->prefetched = c.im && c.tma;
    }

    // The flag lane `lane` of the control warp waits for before the item's
    // M tile is copied (at most one per lane; null when there is none).
    __device__ static const int *producer_flag(const Ctrl &cur, int lane) {
        const ImgDesc &im = *cur.im;
        const int *flag = nullptr;
        if (cur.kind == kItemBand) {
            // the three band+1 tiles this tile reads
            const int c = cur.tile - 1 + lane;
            if (cur.band < im.k - 1 && lane < 3 && c >= 0 && c < im.tiles)
                flag = im.flags + (size_t)(cur.band + 1) * im.tiles + c;
        } else if (cur.kind == kItemDp256) {
            // M(x + d, d), |d| <= 255: band+1 tiles t-4..t+4 (lanes 0..8); the
            // top half at 128-column tile t/2 and the bottom half at t/2-1..t/2+1
            // (lanes 9..12)
            const int ft = cur.tile >> 1;
            if (lane < 9) {
                const int c = cur.tile - 4 + lane;
                if (cur.band < im.k - 1 && c >= 0 && c < im.tiles)
                    flag = im.flags + (size_t)(cur.band + 1) * im.tiles + c;
            } else if (lane == 9) {
                flag = im.fflags + (size_t)(cur.band * 2) * im.ftiles + ft;
            } else if (lane < 13) {
                const int c = ft - 11 + lane;
                if (c >= 0 && c < im.ftiles)
                    flag = im.fflags + (size_t)(cur.band * 2 + 1) * im.ftiles + c;
            }
        }
        return flag;
    }
    // Lanes of the control warp: the item's producer flags, acquired with a
    // bounded spin (true when all are set).
    __device__ static bool wait_producers(const Ctrl &cur, const LaunchArgs &args, int lane) {
        const int *flag = producer_flag(cur, lane);
        bool ok = true;
        if (flag) {
            ok = wait_flag(flag, args.ctl, args.wait_cycles);
            fence_acq_rel_gpu();
        }
        __syncwarp();
        return __all_sync(0xffffffffu, ok);
    }
    // Lanes of the control warp, while the compute warps finish item
    // `busy`: polls the producer flags of the next item until all are set
    // (true; acquired) or the compute warps report `busy` done (false; the
    // flags may then include busy's own, which is published only after it).
    __device__ static bool poll_producers(const Ctrl &nx, const LaunchArgs &args, int lane,
                                          const volatile long long *done, long long busy) {
        const int *flag = producer_flag(nx, lane);
        const long long t0 = clock64();
        for (;;) {
            const bool set = !flag || ld_acquire(flag) != 0;
            if (__all_sync(0xffffffffu, set)) {
                if (flag) fence_acq_rel_gpu();
                __syncwarp();
                return true;
            }
            if (*done == busy || clock64() - t0 > args.wait_cycles ||
                *(volatile const int *)&args.ctl->status != FHTDP_OK)
                return false;
            __nanosleep(64);
        }
    }

    // Items whose M tile may be copied before their FHT ends: F beside the
    // V rows, or no FHT at all (the DP items of 256-row bands).
    __device__ static bool early_copy(const Ctrl &c) {
        return (c.kind == kItemBand && U8Path<Key, true>::early_m(c.n, c.T)) ||
               c.kind == kItemDp256;
    }
    // Lane 0, after the FHT: the M tile of the item into the V rows (or just
    // the arrival on the M barrier when it has none).  Half-band items do
    // not use the M barrier.
    __device__ static void copy_m_tile(const Ctrl &cur, int32_t *Vn, Pipe &pipe) {
        const ImgDesc &im = *cur.im;
        const int n = im.n, D = 2 * n - 1;
        if (cur.kind == kItemHalf0 || cur.kind == kItemHalf1) return;
        if (!im.use_mtma || cur.band >= im.k - 1) {
            mbar_arrive(pipe.mbar);
            return;
        }
        fence_proxy_async_global();
        fence_proxy_async_smem();
        const int y0 = ((cur.band + 1) & 1) * D;
        if (cur.kind == kItemDp256) {
            mbar_expect_tx(pipe.mbar, (uint32_t)(kTile256 * D * 4));
            for (int b = 0; b < D / kMBox256; ++b)
                tma_load_2d(Vn + (kPad + b * kMBox256) * kTile256, &im.mtmap,
                            im.moff + cur.tile * kTile256, y0 + b * kMBox256, pipe.mbar);
            return;
        }
        mbar_expect_tx(pipe.mbar, (uint32_t)(cur.T * D * 4));
        for (int b = 0; b < cur.T / kTile; ++b)
            tma_load_2d(Vn + b * U8Path<Key, true>::vblock(n) + kPad * kTile, &im.mtmap,
                        im.moff + cur.tile * cur.T + b * kTile, y0, pipe.mbar);
    }

    // Lane 0, after the item: its publication (band 0: the tile count, and
    // the read-back after the image's last tile).
    __device__ static void finish(const Ctrl &cur, const LaunchArgs &args) {
        const ImgDesc &im = *cur.im;
        if (cur.kind == kItemHalf0 || cur.kind == kItemHalf1) {
            fence_acq_rel_gpu();
            st_release(im.fflags + (size_t)(cur.band * 2 + cur.kind - kItemHalf0) * im.ftiles +
                           cur.tile,
                       1);
            return;
        }
        const ImgDesc &first_im = args.many ? args.many[0] : args.one;
        if (cur.band != 0) {
            if (!(cur.band == args.skip_band && cur.tile == args.skip_tile &&
                  im.flags == first_im.flags)) {
                fence_acq_rel_gpu();
                st_release(im.flags + (size_t)cur.band * im.tiles + cur.tile, 1);
            }
        } else {
            __threadfence();
            if (atomicAdd(im.done, 1) == im.tiles - 1) readback<int32_t>(im, args);
        }
    }

    // The control warp: takes the items from the queue one ahead of the
    // compute warps, copies each strip as soon as Hc is free, copies an
    // item's M tile as soon as its FHT is done (short bands: as soon as the
    // previous item's window maxima are stored), and releases its flag once its
    // window maxima are stored (band 0: counts the tile and reads the
    // polyline back after the image's last).  The producer flags of the next
    // item are polled while the compute warps finish the current one, so
    // that the M copy seldom waits for them; whatever is not yet set then
    // (possibly the current item's own flag) is waited for after the
    // current item's publication.
    __device__ static void control(const LaunchArgs &args, unsigned char *smem, WsSlot *slot,
                                   Pipe &pipe, const volatile long long *done) {
        const int lane = threadIdx.x & 31;
        uint32_t *Hc = (uint32_t *)(smem + u8_hc_offset<Key>());
        int32_t *Vn = (int32_t *)smem;
        long long idx = 0;
        if (lane == 0) idx = take(args);
        Ctrl cur = decode(args, __shfl_sync(0xffffffffu, idx, 0));
        if (lane == 0) hand_over(cur, slot, Hc, pipe);
        nb_arrive(kBarNext, kCtlSync);
        if (lane == 0 && cur.item < args.items) idx = take(args);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        bool ok = cur.item < args.items ? wait_producers(cur, args, lane) : true;
        bool copied = false;   // cur's M tile is on its way already
        while (cur.item < args.items) {
            // The V rows are free once the previous item's window maxima are
            // stored; where F lies beside them (or there is no FHT) the M
            // copy need not wait for the FHT.  The copy goes out before
            // anything else the control warp does for the item.
            const bool early = early_copy(cur);
            if (early && !copied && lane == 0) {
                if (!ok) atomicExch(&args.ctl->status, FHTDP_ETIMEOUT);
                copy_m_tile(cur, Vn, pipe);
            }
            nb_sync(kBarFhtDone, kCtlSync);
            if (!early && lane == 0) {
                if (!ok) atomicExch(&args.ctl->status, FHTDP_ETIMEOUT);
                copy_m_tile(cur, Vn, pipe);
            }
            const Ctrl next = decode(args, idx);
            nb_sync(kBarHcFree, kCtlSync);
            if (lane == 0) hand_over(next, slot, Hc, pipe);
            nb_arrive(kBarNext, kCtlSync);
            // The item after next is taken now and its index read only after
            // this item's window, so that the queue's round trip overlaps the
            // polling.  A CTA works its items in queue order, so holding one
            // more keeps the queue free of deadlock.
            long long ahead = 0;
            if (lane == 0 && next.item < args.items) ahead = atomicAdd(&args.ctl->queue, 1);
            const bool ready = next.item >= args.items ||
                               poll_producers(next, args, lane, done, cur.item);
            nb_sync(kBarWinDone, kCtlSync);
            // next's producers seen and the V rows free: its M copy goes out
            // before this item's publication.
            copied = ready && next.item < args.items && early_copy(next);
            if (copied && lane == 0) copy_m_tile(next, Vn, pipe);
            if (lane == 0) {
                finish(cur, args);
                if (next.item < args.items) ahead = skip_disabled(args, ahead);
            }
            idx = __shfl_sync(0xffffffffu, ahead, 0);
            ok = ready || wait_producers(next, args, lane);
            cur = next;
        }
    }
};

// ---------------------------------------------------------------------------
// int32 / float images.  Two kinds of work items per band level: FHT items
// compute a band's Hough values for 64 columns, both slope signs, and store
// them to the image's hw rows; DP items of 16 columns bring their Hough rows
// and their M tile by TMA, form V (Eqs. 3-4) as 64-bit window keys, compute
// the bend-window maxima (Sec. 2.3) and publish.  Items are small (256 threads, at
// most 102 KB of shared memory), two CTAs share an SM, and one band level of
// an image spreads over many CTAs, so that the band chain of a single large
// image advances quickly.  The float sums follow the same tree as the
// oracle's float32 recursion (top half + bottom half at every level).
constexpr int kWThreads = 256;
constexpr int kWTileF = 64;    // FHT item columns
constexpr int kWTileD = 16;    // DP item columns
constexpr int kWPad = 48;      // dead rows above and below V in a DP item
constexpr int kItemWideFht = 1, kItemWideDp = 3;

template <typename In, typename Acc, typename Key>
struct WideEngine {
    using KO = KeyOps<Acc, Key>;
    static constexpr int NT = kWThreads;

    __host__ __device__ static int fpitch(int n) { return (kWTileF + n + 8 + 3) & ~3; }
    __host__ __device__ static size_t fht_smem(int n) {
        return (size_t)(n < 2 ? 2 : n) * fpitch(n) * 4;
    }
    // Hough rows [2][n][T] (each sign from a 128-byte boundary, as TMA
    // destinations are), then V [wpad + D + wpad][T]: the M tile lands in its
    // D middle rows and V is formed there in place; the pad rows hold dead
    // values, so that the window reads past [-(n-1), n-1] unchecked.  With a
    // window table, the centred maxima Mc [D + 2 wpad][T] follow.
    __host__ __device__ static int dp_sign1(int n) { return (n * kWTileD + 31) & ~31; }
    __host__ __device__ static size_t dp_mc_off(int n, int wpad) {
        return (size_t)(2 * dp_sign1(n) + (2 * n - 1 + 2 * wpad) * kWTileD) * 4;
    }
    __host__ __device__ static size_t dp_smem(int n, int wpad, bool table) {
        return dp_mc_off(n, wpad) + (table ? (size_t)(2 * n - 1 + 2 * wpad) * kWTileD * 4 : 0);
    }
    static size_t smem_bytes(int max_n, int wpad, bool table) {
        return std::max(fht_smem(max_n), dp_smem(max_n, wpad, table));
    }
    __device__ static Acc *hw_row(const ImgDesc &im, int band, int sign, int s) {
        return (Acc *)im.hw + (((size_t)band * 2 + sign) * im.n + s) * im.hwpitch;
    }

    // Pixels [c, c+4) of a row, zero outside [0, w); c is a multiple of 4.
    __device__ static void load4(const In *row, int c, int w, bool aligned, Acc out[4]) {
        if (aligned && c >= 0 && c + 4 <= w) {
            const int4 v = __ldg((const int4 *)(row + c));
            out[0] = from_bits<Acc>((uint32_t)v.x);
            out[1] = from_bits<Acc>((uint32_t)v.y);
            out[2] = from_bits<Acc>((uint32_t)v.z);
            out[3] = from_bits<Acc>((uint32_t)v.w);
            return;
        }
        for (int j = 0; j < 4; ++j) out[j] = (Acc)pix(row, c + j, w);
    }

    // N consecutive strip words of band row y from word u: sign 0 reads
    // pixels x0 + u.., sign 1 the mirrored strip (word u = pixel x0 + 63 - u).
    template <int N>
    __device__ static void strip_words(const In *row, int w, bool aligned, int x0, int u,
                                       int sign, Acc (&P)[N]) {
        constexpr int NW = (N + 3) / 4;
        Acc q[4 * NW];
        if (sign == 0) {
#pragma unroll
            for (int k = 0; k < NW; ++k) load4(row, x0 + u + 4 * k, w, aligned, &q[4 * k]);
#pragma unroll
            for (int j = 0; j < N; ++j) P[j] = q[j];
        } else {
            // words u .. u + 4NW - 1 are pixels x0 + 63 - u down to x0 + 64 - u - 4NW
            const int c = x0 + kWTileF - u - 4 * NW;
#pragma unroll
            for (int k = 0; k < NW; ++k) load4(row, c + 4 * k, w, aligned, &q[4 * k]);
#pragma unroll
            for (int j = 0; j < N; ++j) P[j] = q[4 * NW - 1 - j];
        }
    }
    // Levels 1 and 2 on four rows y0..y0+3 of a sub-band: out[s][u] (s < 4,
    // u < W) from the rows' words u .. u + W + 2 (the recursion's sums, in
    // its order).
    template <int W>
    __device__ static void levels12(const In *base, long long pitch, int w, bool aligned,
                                    int x0, int u, int sign, int y0, Acc (&out)[4][W]) {
        Acc A[2][W], Bq[2][W + 2];
        {
            Acc p0[W], p1[W + 1];
            strip_words<W>(base + (size_t)y0 * pitch, w, aligned, x0, u, sign, p0);
            strip_words<W + 1>(base + (size_t)(y0 + 1) * pitch, w, aligned, x0, u, sign, p1);
#pragma unroll
            for (int j = 0; j < W; ++j) {
                A[0][j] = p0[j] + p1[j];
                A[1][j] = p0[j] + p1[j + 1];
            }
        }
        {
            Acc p2[W + 2], p3[W + 3];
            strip_words<W + 2>(base + (size_t)(y0 + 2) * pitch, w, aligned, x0, u, sign, p2);
            strip_words<W + 3>(base + (size_t)(y0 + 3) * pitch, w, aligned, x0, u, sign, p3);
#pragma unroll
            for (int j = 0; j < W + 2; ++j) {
                Bq[0][j] = p2[j] + p3[j];
                Bq[1][j] = p2[j] + p3[j + 1];
            }
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            out[0][j] = A[0][j] + Bq[0][j];
            out[1][j] = A[0][j] + Bq[0][j + 1];
            out[2][j] = A[1][j] + Bq[1][j + 1];
            out[3][j] = A[1][j] + Bq[1][j + 2];
        }
    }
    // Levels 1-3 in registers straight from the image (n >= 8): a task is an
    // 8-row sub-band g and the 4 words [4c, 4c + 4) of the level-3 width;
    // shift s of the sub-band goes to row 8g + brev3(s) of F.
    __device__ static void fht_regs8(Acc *F, int pitch, const ImgDesc &im, const In *base,
                                     bool aligned, int x0, int sign) {
        const int n = im.n, T = kWTileF;
        const int C4 = (T + n - 8 + 3) / 4;
        const int tasks = (n / 8) * C4;
        for (int t = threadIdx.x; t < tasks; t += NT) {
            const int g = t / C4, c = t - g * C4;
            Acc B2[4][8], T2[4][4];
            levels12<8>(base, im.pitch, im.w, aligned, x0, 4 * c, sign, 8 * g + 4, B2);
            levels12<4>(base, im.pitch, im.w, aligned, x0, 4 * c, sign, 8 * g, T2);
            Acc *row0 = F + (size_t)(8 * g) * pitch + 4 * c;
#pragma unroll
            for (int sh = 0; sh < 8; ++sh) {
                const int h = sh >> 1, o = (sh + 1) >> 1;
                const int r = ((sh & 1) << 2) | (sh & 2) | ((sh >> 2) & 1);
                *(uint4 *)&row0[(size_t)r * pitch] =
                    make_uint4(to_bits(T2[h][0] + B2[h][o + 0]), to_bits(T2[h][1] + B2[h][o + 1]),
                               to_bits(T2[h][2] + B2[h][o + 2]), to_bits(T2[h][3] + B2[h][o + 3]));
            }
        }
        csync<NT>();
    }

    // FHT item: the band's Hough values of columns [x0, x0 + 64), both signs,
    // into hw.  Sign 0 ("+") runs on the strip as it is and its last level
    // writes the rows of hw directly; sign 1 ("-") runs on the mirrored strip
    // (word u = pixel x0 + 63 - u), and its rows, bit-reversed in F, are
    // copied out mirrored back.
    // The strip of an FHT item (columns [x0, x0 + T + n - 1) of the band's
    // rows, clipped to the image) requested into L2, every 128-byte line at
    // once, at the item's start: the register levels read the strip task by
    // task, and their first reads would otherwise wait on DRAM one task
    // after another.
    __device__ static void prefetch_strip(const ImgDesc &im, int band, int ft) {
        const int n = im.n, x0 = ft * kWTileF;
        const In *base = (const In *)im.img + (size_t)band * n * im.pitch;
        const int c_lo = x0, c_hi = min(x0 + kWTileF + n - 1, im.w);   // [c_lo, c_hi)
        if (c_lo >= c_hi) return;
        const size_t bytes = (size_t)(c_hi - c_lo) * sizeof(In);
        const int lines = (int)((bytes + 127) / 128) + 1;
        for (int i = threadIdx.x; i < n * lines; i += NT) {
            const int y = i / lines, l = i - y * lines;
            const uintptr_t a = (uintptr_t)(base + (size_t)y * im.pitch + c_lo);
            const uintptr_t line = (a & ~(uintptr_t)127) + (uintptr_t)l * 128;
            // only lines that hold a byte of the row's range
            if (line < a + bytes) prefetch_l2((const void *)line);
        }
    }

    __device__ static void fht_item(const ImgDesc &im, int band, int ft, unsigned char *smem) {
        const int n = im.n, T = kWTileF, pitch = fpitch(n), x0 = ft * T;
        Acc *F = (Acc *)smem;
        const int G = (T + n - 1 + 3) / 4;
        const In *base = (const In *)im.img + (size_t)band * n * im.pitch;
        const bool aligned = ((uintptr_t)im.img % 16 == 0) && (im.pitch % 4 == 0);
        constexpr int kLB = 8;
        prefetch_strip(im, band, ft);
        for (int sign = 0; sign < 2; ++sign) {
            int first = 1;   // the first level left to merge in shared memory
            if (n >= 8) {
                fht_regs8(F, pitch, im, base, aligned, x0, sign);
                first = 4;
            } else
            for (int b0 = threadIdx.x; b0 < n * G; b0 += kLB * NT) {
                Acc v[kLB][4];
#pragma unroll
                for (int i = 0; i < kLB; ++i) {
                    const int idx = b0 + i * NT;
                    if (idx < n * G) {
                        const int y = idx / G, u0 = 4 * (idx - y * G);
                        load4(base + (size_t)y * im.pitch, sign == 0 ? x0 + u0 : x0 + T - 4 - u0,
                              im.w, aligned, v[i]);
                    }
                }
#pragma unroll
                for (int i = 0; i < kLB; ++i) {
                    const int idx = b0 + i * NT;
                    if (idx < n * G) {
                        const int y = idx / G, u0 = 4 * (idx - y * G);
                        const bool fw = sign == 0;
                        *(uint4 *)&F[(size_t)y * pitch + u0] =
                            make_uint4(to_bits(fw ? v[i][0] : v[i][3]),
                                       to_bits(fw ? v[i][1] : v[i][2]),
                                       to_bits(fw ? v[i][2] : v[i][1]),
                                       to_bits(fw ? v[i][3] : v[i][0]));
                    }
                }
            }
            csync<NT>();
            if (sign == 0) {
                if (!fht_merge<Acc, NT>(F, pitch, n, im.log2n, T, first,
                                         hw_row(im, band, 0, 0) + x0, im.hwpitch)) {
                    // no merge level (n = 1, or n = 8 done in registers): rows
                    // brev(s) hold the shifts
                    for (int idx = threadIdx.x; idx < n * T; idx += NT) {
                        const int sh = idx / T, u = idx - sh * T;
                        hw_row(im, band, 0, sh)[x0 + u] = F[(size_t)brev(sh, im.log2n) * pitch + u];
                    }
                }
            } else {
                fht_merge<Acc, NT>(F, pitch, n, im.log2n, T, first);
                // shift s of the mirrored strip at word u: the left-moving sum
                // from column x0 + 63 - u, in row brev(s) of F
                for (int idx = threadIdx.x; idx < n * (T / 4); idx += NT) {
                    const int sh = idx / (T / 4), u0 = 4 * (idx % (T / 4));
                    const uint4 w4 =
                        *(const uint4 *)&F[(size_t)brev(sh, im.log2n) * pitch + T - 4 - u0];
                    *(uint4 *)(hw_row(im, band, 1, sh) + x0 + u0) =
                        make_uint4(w4.w, w4.z, w4.y, w4.x);
                }
            }
            csync<NT>();
        }
    }

    // DP item: columns [x0, x0 + 16) of band `band`.
    __device__ static void dp_item(const ImgDesc &im, int band, int tile, unsigned char *smem,
                                   Pipe &pipe, const LaunchArgs &args) {
        const int n = im.n, D = 2 * n - 1, T = kWTileD, x0 = tile * T;
        const bool last = band == im.k - 1;
        const int wpad = args.wpad;
        Acc *Ht = (Acc *)smem;          // [2][n][T]: Hough rows of both signs
        const int h1 = dp_sign1(n);     // offset of sign 1
        Acc *Vt = Ht + 2 * h1;          // [wpad + D + wpad][T]: M tile, then V
        Acc *Mt = Vt + wpad * T;        // row e + n - 1: displacement e
        const Acc dead = Dead<Acc>::value();
        if (threadIdx.x < 32) {
            // M(x + d, d): band+1 tiles over [x0 - (n-1), x0 + T + n - 2] (lanes
            // 0..30); the FHT item of these columns (lane 31)
            const int lane = threadIdx.x;
            const int t0 = (x0 - (n - 1)) >= 0 ? (x0 - (n - 1)) / T : -((n - 1 - x0 + T - 1) / T);
            const int *flag = nullptr;
            if (lane < 31) {
                const int c = t0 + lane;
                if (!last && c >= 0 && c < im.tiles && c * T <= x0 + T + n - 2)
                    flag = im.flags + (size_t)(band + 1) * im.tiles + c;
            } else {
                flag = im.fflags + (size_t)band * im.ftiles + x0 / kWTileF;
            }
            bool ok = true;
            if (flag) {
                ok = wait_flag(flag, args.ctl, args.wait_cycles);
                fence_acq_rel_gpu();
            }
            __syncwarp();
            ok = __all_sync(0xffffffffu, ok);
            if (lane == 0) {
                if (!ok) atomicExch(&args.ctl->status, FHTDP_ETIMEOUT);
                fence_proxy_async_global();
                fence_proxy_async_smem();
                mbar_expect_tx(pipe.mbar, (uint32_t)((2 * n + (last ? 0 : D)) * T * 4));
                tma_load_2d(Ht, &im.tmap, x0, band * 2 * n, pipe.mbar);
                tma_load_2d(Ht + h1, &im.tmap, x0, (band * 2 + 1) * n, pipe.mbar);
                if (!last) tma_load_2d(Mt, &im.mtmap, im.moff + x0, (band + 1) * D, pipe.mbar);
            }
        } else if (band != 0) {
            // the dead pad rows (outside the copies' destinations)
            for (int idx = threadIdx.x - 32; idx < 2 * wpad * (T / 4); idx += NT - 32) {
                const int r = idx / (T / 4), u0 = 4 * (idx % (T / 4));
                const int row = r < wpad ? r : r + D;
                *(uint4 *)&Vt[row * T + u0] =
                    make_uint4(to_bits(dead), to_bits(dead), to_bits(dead), to_bits(dead));
            }
        }
        if (!mbar_wait(pipe.mbar, pipe.mphase, args.wait_cycles)) {
            if (threadIdx.x == 0) atomicExch(&args.ctl->status, FHTDP_ETIMEOUT);
            mbar_wait(pipe.mbar, pipe.mphase, kDrainCycles);
        }
        pipe.mphase ^= 1u;
        // V(x, e) = H(x, e) + M(x + e, e), dead outside the image (Eqs. 3-4),
        // in place of the M tile.
        unsigned long long best = 0;
        for (int idx = threadIdx.x; idx < D * (T / 4); idx += NT) {
            const int ei = idx / (T / 4), u0 = 4 * (idx % (T / 4));
            const int e = ei - (n - 1), sh = e < 0 ? -e : e;
            const uint4 h4 = *(const uint4 *)&Ht[(e < 0 ? h1 : 0) + sh * T + u0];
            uint4 m4 = make_uint4(0, 0, 0, 0);
            if (!last) m4 = *(const uint4 *)&Mt[ei * T + u0];
            const uint32_t hb[4] = {h4.x, h4.y, h4.z, h4.w};
            const uint32_t mb[4] = {m4.x, m4.y, m4.z, m4.w};
            Acc v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int x = x0 + u0 + j;
                const bool ok = x < im.w && x + e >= 0 && x + e < im.w;
                const Acc h = from_bits<Acc>(hb[j]), m = from_bits<Acc>(mb[j]);
                v[j] = !ok ? dead : last ? h : (m == dead ? dead : h + m);
            }
            if (band == 0) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (v[j] != dead) {
                        const unsigned long long k = argmax_key(ord32(v[j]), x0 + u0 + j, ei);
                        best = best > k ? best : k;
                    }
            } else {
                *(uint4 *)&Mt[ei * T + u0] =
                    make_uint4(to_bits(v[0]), to_bits(v[1]), to_bits(v[2]), to_bits(v[3]));
            }
        }
        if (band == 0) {
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
                best = best > other ? best : other;
            }
            if ((threadIdx.x & 31) == 0 && best) atomicMax(im.best, best);
            csync<NT>();
            if (threadIdx.x < 32) {
                int is_last = 0;
                if (threadIdx.x == 0) {
                    __threadfence();
                    is_last = atomicAdd(im.done, 1) == im.tiles - 1;
                }
                if (__shfl_sync(0xffffffffu, is_last, 0)) readback_values(im, args);
            }
            return;
        }
        csync<NT>();
        // Window maxima (values only: the read-back recomputes the argmax),
        // 16 threads per column, 16 displacements each.
        const int u = threadIdx.x & (T - 1), q = threadIdx.x / T;
        const int x = x0 + u;
        const int lo = -(n - 1), hi = n - 1;
        const int B = args.use_table ? args.B0 : im.B;
        const Acc *col = Mt + (n - 1) * T + u;   // V(e) at col[e * T]
        // Runs of NOUT outputs from c0 (count of them) of the maxima over
        // [c - B, c + B], NOUT the largest power of two up to 16 that the
        // window length L = 2B + 1 covers (one block pair per run).
        auto maxima = [&](int c0, int count, auto vkey, auto emit) {
            auto runs = [&](auto nout) {
                constexpr int NOUT = decltype(nout)::value;
                for (int r0 = 0; r0 < count; r0 += NOUT)
                    window_span<NOUT, Acc>(c0 + r0, count - r0, B, dead, vkey,
                                           [&](int i, Acc m) { emit(r0 + i, m); });
            };
            const int L = 2 * B + 1;
            if (L >= 16) runs(std::integral_constant<int, 16>());
            else if (L >= 8) runs(std::integral_constant<int, 8>());
            else if (L >= 4) runs(std::integral_constant<int, 4>());
            else if (L >= 2) runs(std::integral_constant<int, 2>());
            else runs(std::integral_constant<int, 1>());
        };
        auto vpad = [&](int e) -> Acc { return col[e * T]; };   // dead pad rows outside
        const int c0 = lo + 16 * q;
        if (!args.use_table) {
            if (x < im.w && c0 <= hi) {
                Acc *mcol = mband(im, band) + (size_t)(c0 + n - 1) * im.mpitch + im.moff + x - c0;
                const int count = min(16, hi - c0 + 1);
                auto emit = [&](int i, Acc m) { mcol[(long long)i * (im.mpitch - 1)] = m; };
                // A run reads V over [c - B, c + B + 16]: inside the pad rows
                // when B + 16 <= wpad.
                if (B + 16 <= wpad) maxima(c0, count, vpad, emit);
                else
                    maxima(c0, count,
                           [&](int e) -> Acc { return (e < lo || e > hi) ? dead : col[e * T]; },
                           emit);
            }
        } else {
            // Bend-angle windows (Sec. 2.3): the centred maxima Mc(p) over
            // [p - B0, p + B0] for p in [-(n-1) - B0, n-1 + B0] (they read V
            // over [-(n-1) - 2 B0, n-1 + 2 B0 + 16], inside the pad rows),
            // then each window [lo(c), hi(c)] as the maximum of the pieces
            // that cover it: centres lo + B0, lo + B0 + L, ... and hi - B0.  A
            // window shorter than L = 2 B0 + 1 is cut by an end of the range:
            // the piece from its other end reaches only dead rows beyond it.
            Acc *Mc = (Acc *)(smem + dp_mc_off(n, wpad)) + u;   // row p + (n-1) + B0
            const int NC = D + 2 * B;
            for (int i0 = 16 * q; i0 < NC; i0 += 16 * (NT / T))
                maxima(i0 - (n - 1) - B, min(16, NC - i0), vpad,
                       [&](int i, Acc m) { Mc[(size_t)(i0 + i) * T] = m; });
            csync<NT>();
            if (x < im.w && c0 <= hi) {
                Acc *mcol = mband(im, band) + (size_t)(c0 + n - 1) * im.mpitch + im.moff + x - c0;
                const int count = min(16, hi - c0 + 1);
                const int L = 2 * B + 1;
                auto mc = [&](int p) -> Acc { return Mc[(size_t)(p + n - 1 + B) * T]; };
                for (int i = 0; i < count; ++i) {
                    const int c = c0 + i;
                    const int wl = args.tab.lo[c + n - 1], wh = args.tab.hi[c + n - 1];
                    Acc m = dead;
                    if (wh - wl + 1 >= L) {
                        for (int p = wl + B; p < wh - B; p += L) m = kmax(m, mc(p));
                        m = kmax(m, mc(wh - B));
                    } else if (wh == hi) {
                        m = mc(wl + B);
                    } else if (wl == lo) {
                        m = mc(wh - B);
                    } else {   // not produced by the host's choice of B0; kept exact
                        for (int e = wl; e <= wh; ++e) m = kmax(m, col[e * T]);
                    }
                    mcol[(long long)i * (im.mpitch - 1)] = m;
                }
            }
        }
        fence_acq_rel_gpu();
        csync<NT>();
        if (threadIdx.x == 0) {
            const ImgDesc &first = args.many ? args.many[0] : args.one;
            if (!(band == args.skip_band && tile == args.skip_tile && im.flags == first.flags))
                st_release(im.flags + (size_t)band * im.tiles + tile, 1);
        }
    }

    // The window maxima of band b: [D][mpitch], one array per band (the
    // read-back recomputes each band's argmax from them and the Hough rows).
    __device__ static Acc *mband(const ImgDesc &im, int band) {
        return (Acc *)im.mbuf[0] + (size_t)band * (2 * im.n - 1) * im.mpitch;
    }

    // Eq. 5 by one warp, from the best top point: at band i the smallest e
    // with |e - d_{i-1}| <= B maximising V_i(x_i, e) = H_i(x_i, e) +
    // M_{i+1}(x_i + e, e), recomputed from the stored Hough rows and window
    // maxima with the same additions as the DP item (lanes over e, then a
    // warp maximum of (value, smallest e) keys).
    __device__ static void readback_values(const ImgDesc &im, const LaunchArgs &args) {
        const int lane = threadIdx.x & 31, n = im.n, D = 2 * n - 1;
        const Acc dead = Dead<Acc>::value();
        __threadfence();
        unsigned long long key = 0;
        if (lane == 0) key = atomicAdd(im.best, 0ull);
        key = __shfl_sync(0xffffffffu, key, 0);
        if (key == 0) {   // no admissible polyline
            if (lane == 0) {
                *(Acc *)im.score_out = dead;
                for (int i = 0; i <= im.k; ++i) im.x_out[i] = -1;
                for (int i = 0; i < im.k; ++i) im.d_out[i] = 0;
            }
            return;
        }
        const unsigned lin = 0xffffffffu - (unsigned)(key & 0xffffffffu);
        int xx = (int)(lin >> 9), d = (int)(lin & 511) - (n - 1);
        if (lane == 0) {
            im.x_out[0] = xx;
            im.d_out[0] = d;
            *(Acc *)im.score_out = from_ord32<Acc>((uint32_t)(key >> 32));
        }
        for (int i = 1; i < im.k; ++i) {
            xx += d;
            // Only reachable with inconsistent DP data (a wait gave up): stop
            // instead of reading outside the arrays.
            if (xx < 0 || xx >= im.w || d < -(n - 1) || d > n - 1) {
                if (lane == 0) atomicExch(&args.ctl->status, FHTDP_ETIMEOUT);
                return;
            }
            const int lo = args.use_table ? args.tab.lo[d + n - 1] : max(-(n - 1), d - im.B);
            const int hi = args.use_table ? args.tab.hi[d + n - 1] : min(n - 1, d + im.B);
            const Acc *mb = i + 1 < im.k ? mband(im, i + 1) : nullptr;
            unsigned long long bk = 0;
            for (int e = lo + lane; e <= hi; e += 32) {
                const int sh = e < 0 ? -e : e;
                Acc v = dead;   // the link must end inside the image (every band)
                if (xx + e >= 0 && xx + e < im.w) {
                    const Acc h =
                        from_bits<Acc>(__ldcg((const uint32_t *)hw_row(im, i, e < 0, sh) + xx));
                    v = h;
                    if (mb) {
                        // M_{i+1}(xx + e, e): row e + n - 1, skewed column moff + xx
                        const Acc m = from_bits<Acc>(__ldcg(
                            (const uint32_t *)mb + (size_t)(e + n - 1) * im.mpitch + im.moff + xx));
                        v = m == dead ? dead : h + m;
                    }
                }
                if (v != dead) {
                    const unsigned long long k =
                        ((unsigned long long)ord32(v) << 32) | (0xffffffffu - (unsigned)(e + n - 1));
                    bk = bk > k ? bk : k;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, bk, o);
                bk = bk > other ? bk : other;
            }
            if (bk == 0) {   // inconsistent data, as above
                if (lane == 0) atomicExch(&args.ctl->status, FHTDP_ETIMEOUT);
                return;
            }
            d = (int)(0xffffffffu - (unsigned)(bk & 0xffffffffu)) - (n - 1);
            if (lane == 0) {
                im.x_out[i] = xx;
                im.d_out[i] = d;
            }
        }
        if (lane == 0) im.x_out[im.k] = xx + d;
    }
};

// The work items of an image whose bands need FHT items of their own (int32
// / float images; the half-band items of 256-row uint8 bands), in queue
// order, by band level: level 0 opens with the FHT items of band k-1; level
// lv (band b = k-1-lv) holds the DP items of band b and, spread evenly among
// them (or in a block before them), the FHT items of band b - A (level 0: of
// bands k-2 .. k-1-A).  An FHT
// item takes several DP items' time, so it is queued A levels before the DP
// items that read its rows, and spreading them keeps a level's DP items from
// waiting behind a block of FHT items.  Every item still comes after all the
// items it waits for.
constexpr int kWAhead = 2;
struct WideLevels {
    int k;
    long long F, P;   // FHT and DP items of one band
    int A = kWAhead;  // levels between an FHT item and the DP items that read it
    bool spread = true;   // false: a level's FHT items before its DP items
    __host__ __device__ long long fht_in(int lv) const {   // FHT items spread in level lv
        if (lv == 0) return (long long)(A < k - 1 ? A : k - 1) * F;
        return k - 1 - lv - A >= 0 ? F : 0;
    }
    // First item of level lv (lv = k: the item count).
    __host__ __device__ long long start(int lv) const {
        if (lv == 0) return 0;
        const long long l0 = F + fht_in(0) + P;
        int full = lv - 1 < k - 1 - A ? lv - 1 : k - 1 - A;   // levels 1.. with F
        if (full < 0) full = 0;
        return l0 + (long long)full * (F + P) + (long long)(lv - 1 - full) * P;
    }
    // Item `off` of level lv: FHT item `tile` of `band` (kind 0), or DP item
    // `tile` of `band` (kind 1).
    __host__ __device__ void at(int lv, long long off, int *kind, int *band, int *tile) const {
        const int b = k - 1 - lv;
        if (lv == 0) {
            if (off < F) {
                *kind = 0;
                *band = k - 1;
                *tile = (int)off;
                return;
            }
            off -= F;
        }
        const long long Fl = fht_in(lv), S = Fl + P;
        const long long c0 = spread ? off * Fl / S : (off < Fl ? off : Fl);
        const long long c1 = spread ? (off + 1) * Fl / S : (off < Fl ? off + 1 : Fl);
        if (c1 > c0) {   // the FHT item number c0 of the level
            *kind = 0;
            *band = lv == 0 ? k - 2 - (int)(c0 / F) : b - A;
            *tile = (int)(c0 % F);
        } else {
            *kind = 1;
            *band = b;
            *tile = (int)(off - c0);
        }
    }
    __host__ __device__ void decode(long long item, int *kind, int *band, int *tile) const {
        int lo = 0, hi = k - 1;   // the last level that starts at or before item
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (start(mid) <= item) lo = mid;
            else hi = mid - 1;
        }
        at(lo, item - start(lo), kind, band, tile);
    }
};

__device__ inline void decode_wide_one(const ImgDesc &im, long long item, int *kind, int *band,
                                       int *tile) {
    int fd;
    WideLevels{im.k, im.ftiles, im.tiles}.decode(item, &fd, band, tile);
    *kind = fd ? kItemWideDp : kItemWideFht;
}

template <typename In, typename Acc, typename Key>
__global__ void __launch_bounds__(kWThreads, 2)
    engine_kernel_wide(const __grid_constant__ LaunchArgs args) {
    using P = WideEngine<In, Acc, Key>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ long long s_item;
    if (threadIdx.x == 0) {
        mbar_init(&s_mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    Pipe pipe{nullptr, 0u, &s_mbar, 0u, nullptr};
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&args.ctl->queue, 1);
        csync<kWThreads>();
        const long long item = s_item;
        csync<kWThreads>();   // s_item is rewritten at the next item
        if (item >= args.items) break;
        const ImgDesc *im;
        int kind, band, tile;
        if (args.many) {
            const Item it = args.order[item];
            im = &args.many[it.image];
            kind = (it.nflags >> 19) & 3;
            band = it.band;
            tile = it.tile;
        } else {
            im = &args.one;
            decode_wide_one(args.one, item, &kind, &band, &tile);
        }
        if (kind == kItemWideFht) {
            P::fht_item(*im, band, tile, smem_raw);
            if (threadIdx.x == 0) {
                fence_acq_rel_gpu();
                st_release(im->fflags + (size_t)band * im->ftiles + tile, 1);
            }
        } else {
            P::dp_item(*im, band, tile, smem_raw, pipe, args);
        }
    }
}

// The uint8 engine: four compute warpgroups (112 registers a thread) and a
// control warp (32 registers; the rest of its warpgroup exits at once).  The
// register split adds up to the launch's 640 x 96.
template <typename Key, bool kMulti>
__global__ void __launch_bounds__(kWsThreads, 1)
    engine_kernel_u8(const __grid_constant__ LaunchArgs args) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ __align__(16) WsSlot s_slot;
    __shared__ volatile long long s_done;   // the last item thread 0 finished
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1);
        mbar_init(&s_mbar, 1);
        s_done = -1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    Pipe pipe{&s_bar, 0u, &s_mbar, 0u, nullptr};
    if (threadIdx.x < kThreads) {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 112;" ::: "memory");
        for (;;) {
            nb_sync(kBarNext, kCtlSync);
            const WsSlot sl = s_slot;
            if (sl.item >= args.items) break;
            if constexpr (kMulti) {
                if (sl.kind == kItemDp256) {
                    U8Path<Key, kMulti>::process_dp256(*sl.im, sl.band, sl.tile, smem_raw, args,
                                                       pipe);
                    if (threadIdx.x == 0) s_done = sl.item;
                    continue;
                }
            }
            const int half = sl.kind == kItemHalf0 ? 0 : sl.kind == kItemHalf1 ? 1 : -1;
            U8Path<Key, kMulti>::process(*sl.im, sl.band, sl.tile, smem_raw, args, pipe,
                                         sl.prefetched != 0, half);
            // a hint for the control warp's polling (ordering comes from kBarWinDone)
            if (threadIdx.x == 0) s_done = sl.item;
        }
    } else {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 32;" ::: "memory");
        if (threadIdx.x < kCtlSync) U8Ctl<Key>::control(args, smem_raw, &s_slot, pipe, &s_done);
    }
}

// ---------------------------------------------------------------------------
// Host side.
//
// Workspace of a run: [Ctl][per-image counters: flags, best, done][image
// table][per-image M ping-pong buffers and backpointers].  The first two
// parts are cleared by one memset per run; the table is written once by
// fhtdp_batch_upload (single-image runs pass their descriptor by value).
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct ImgPlan {
    fhtdp_image io;
    Shape s;
    int B, tiles, mpitch;
    int T;                      // column tile width of its work items
    int depth;                  // uint8: FHT levels in registers (2 or 3)
    int kind;                   // 1: 256-row bands through half-band and DP items
    int ftiles, hpitch, moff;   // kind 1: half-band tiles, h256 row pitch; M column offset
    const int32_t *enable;      // optional: the image runs only where this reads nonzero
    int mask1, mask_x, mask_end;   // optional point of Subproblems 2-3 (see ImgDesc)
    long long item0;
    size_t flags, best, done, fflags;   // offsets in the counter region
    size_t m0, m1, bp, h256;            // offsets in the data region
};

struct RunLayout {
    size_t zero_bytes;   // Ctl + counters
    size_t table_off, table_bytes;
    size_t order_off, order_bytes;
    size_t data_off, total;
    long long items;
    int max_n, max_h;
    bool multi_tile;     // some image's tiles are not kTile wide
};

// Column tile width of an image's work items: uint8 images with bands of at
// most 64 rows take 256 columns (more work per item and fewer items for the
// short bands), the others 128.
int default_tile(int dtype, int n) { return dtype == FHTDP_U8 && n <= 64 ? 256 : kTile; }

int tiles_of(const Shape &s, int T) { return (s.w + T - 1) / T; }

// uint8 images with 256-row bands run in the fused engine when their strips
// can go through TMA (16-byte aligned rows) and the backpointer byte
// identifies the argmax inside a window (B <= 127); the others take the
// standalone kernels.
bool fused_256(int dtype, const Shape &s, int B, const void *img, long long pitch) {
    return dtype == FHTDP_U8 && s.n == 256 && B <= 127 && (uintptr_t)img % 16 == 0 &&
           pitch % 16 == 0;
}
// Queue-entry code of a tile width: T = 64 << code.
int tile_code(int T) { return T == 256 ? 2 : T == 64 ? 0 : 1; }

// Tile widths a uint8 image's items may take (the tuner's choices): bands of
// at most 64 rows 128 or 256, 128-row bands 128, 256-row bands 64.
bool tile_choice(int dtype, const ImgPlan &p, int T) {
    if (dtype != FHTDP_U8 || p.kind == 1) return T == p.T;
    return T == kTile || (T == 2 * kTile && p.s.n <= max_band<2 * kTile>());
}

// With `reserve`, every image's counters and buffers are sized for the
// largest of its tile-width choices (most tiles, widest M rows), so that the
// workspace fits any choice the tuner makes.
RunLayout plan_layout(std::vector<ImgPlan> &imgs, bool with_table, bool reserve = false,
                      int dtype = FHTDP_U8) {
    RunLayout L{};
    size_t off = sizeof(Ctl);
    long long items = 0;
    for (auto &p : imgs) {
        const int T0 = p.T;
        if (reserve && tile_choice(dtype, p, kTile)) p.T = kTile;   // the most tiles
        p.tiles = tiles_of(p.s, p.T);
        if (reserve && tile_choice(dtype, p, 2 * kTile)) p.T = 2 * kTile;   // the widest rows
        p.item0 = items;
        items += (long long)p.s.k * p.tiles;
        if (p.kind == 1) {
            // M(x', c) at column moff + x' - c, |c| <= 255; the M tile reads
            // go up to 64 words past the last tile's columns.
            p.moff = 256;
            p.mpitch = (int)align_up((size_t)p.moff + p.s.w + 256 + 4, 32);
            p.ftiles = (p.s.w + kTile - 1) / kTile;
            p.hpitch = kH256Left + p.ftiles * kTile + kH256Right;
            items += 2LL * p.s.k * p.ftiles;
            p.fflags = off;
            off = align_up(off + (size_t)p.s.k * 2 * p.ftiles * 4, 8);
        } else if (p.kind == 2) {
            p.moff = kMOff;
            p.mpitch = (int)align_up((size_t)kMOff + p.s.w + kWTileD + 4, 32);
            p.ftiles = (p.s.w + kWTileF - 1) / kWTileF;
            p.hpitch = p.ftiles * kWTileF;
            items += (long long)p.s.k * p.ftiles;
            p.fflags = off;
            off = align_up(off + (size_t)p.s.k * p.ftiles * 4, 8);
        } else {
            // Row reads of M go up to 4 words past the last tile's columns.
            p.moff = kMOff;
            p.mpitch = (int)align_up((size_t)kMOff + p.s.w + p.T + 4, 32);
        }
        p.T = T0;
        p.flags = off;
        off = align_up(off + (size_t)p.s.k * p.tiles * 4, 8);
        p.best = off;
        off += 8;
        p.done = off;
        off = align_up(off + 4, 8);
        L.max_n = std::max(L.max_n, p.s.n);
        if (p.T != kTile) L.multi_tile = true;
        L.max_h = std::max(L.max_h, p.s.h);
    }
    L.zero_bytes = align_up(off, 256);
    L.table_off = L.zero_bytes;
    L.table_bytes = with_table ? align_up(sizeof(ImgDesc) * imgs.size(), 256) : 0;
    L.order_off = L.table_off + L.table_bytes;
    L.order_bytes = with_table ? align_up(sizeof(Item) * (size_t)items, 256) : 0;
    size_t d = 0;
    for (auto &p : imgs) {
        p.m0 = d;   // the two M buffers are adjacent: one tensor map covers both
        if (p.kind == 2) {
            // int32 / float images: one M array per band and no backpointers
            // (the read-back recomputes each band's argmax)
            p.m1 = d;
            d = align_up(d + (size_t)p.s.k * p.s.D * p.mpitch * 4, 256);
            p.bp = d;
        } else {
            p.m1 = d + (size_t)p.s.D * p.mpitch * 4;
            d = align_up(p.m1 + (size_t)p.s.D * p.mpitch * 4, 256);
            p.bp = d;
            d = align_up(d + (size_t)p.s.k * bp_groups(p.s.n) * 4 * p.s.w, 256);
        }
        if (p.kind == 1) {
            p.h256 = d;
            d = align_up(d + (size_t)p.s.k * 4 * 128 * p.hpitch * 2, 256);
        } else if (p.kind == 2) {
            p.h256 = d;   // the Hough rows, [k][2][n][hpitch] of 4 bytes
            d = align_up(d + (size_t)p.s.k * 2 * p.s.n * p.hpitch * 4, 256);
        }
    }
    L.data_off = L.order_off + L.order_bytes;
    L.total = L.data_off + d;
    L.items = items;
    return L;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link-time dependency on the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D uint8 tensor map of an image, box of 128 columns x n rows, zero fill
// outside the image.  False when the image cannot be described (the strip is
// then read with plain loads).
bool encode_strip_map(CUtensorMap *map, const void *img, int h, int w, long long pitch, int n) {
    if ((uintptr_t)img % 16 != 0 || pitch % 16 != 0 || n < 4 || n > 256) return false;
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t strides[1] = {(cuuint64_t)pitch};
    // 256-row bands are staged one 128-row half at a time.
    cuuint32_t box[2] = {128u, (cuuint32_t)(n > 128 ? 128 : n)};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(img), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D int32 tensor map of an image's adjacent M buffers ([arrays * D][mpitch]:
// two ping-pong buffers, or one per band for int32 / float images), box of bw
// columns x bh rows: for uint8 bands of at most 128 rows 128 x D (one copy
// brings a tile's whole M_{b+1}), for 256-row bands 64 x 73 (seven), for
// int32 / float images 16 x D.
bool encode_m_map(CUtensorMap *map, void *m0, int D, int mpitch, int bw, int bh,
                  int arrays = 2) {
    if ((uintptr_t)m0 % 16 != 0 || mpitch % 4 != 0 || bh > 256 || bw > 256) return false;
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)mpitch, (cuuint64_t)arrays * D};
    cuuint64_t strides[1] = {(cuuint64_t)mpitch * 4};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, m0, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D tensor map of `rows` rows of `pitch` 4-byte values, box bw x bh (the
// Hough rows of an int32 / float image).
bool encode_rows_map(CUtensorMap *map, void *base, int pitch, int rows, int bw, int bh) {
    if ((uintptr_t)base % 16 != 0 || pitch % 4 != 0 || bh > 256 || bw > 256) return false;
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

ImgDesc make_desc(const ImgPlan &p, const RunLayout &L, char *ws, int dtype) {
    ImgDesc im{};
    im.use_tma = dtype == FHTDP_U8 &&
                 encode_strip_map(&im.tmap, p.io.img, p.s.h, p.s.w, p.io.pitch, p.s.n);
    // (int32 / float images: tmap describes their Hough rows, below)
    if (p.kind == 1)
        im.use_mtma = ws && encode_m_map(&im.mtmap, ws + L.data_off + p.m0, p.s.D, p.mpitch,
                                         kTile256, kMBox256);
    else if (p.kind == 2)
        im.use_mtma = ws && encode_m_map(&im.mtmap, ws + L.data_off + p.m0, p.s.D, p.mpitch,
                                         kWTileD, p.s.D, p.s.k) &&
                      encode_rows_map(&im.tmap, ws + L.data_off + p.h256, p.hpitch,
                                      2 * p.s.k * p.s.n, kWTileD, p.s.n);
    else
        im.use_mtma = dtype == FHTDP_U8 && p.s.n <= kMaxBandFused && ws &&
                      encode_m_map(&im.mtmap, ws + L.data_off + p.m0, p.s.D, p.mpitch, kTile,
                                   p.s.D);
    im.img = p.io.img;
    im.pitch = p.io.pitch;
    im.h = p.s.h;
    im.w = p.s.w;
    im.k = p.s.k;
    im.n = p.s.n;
    im.log2n = p.s.log2n;
    im.B = p.B;
    im.tiles = p.tiles;
    im.tw = p.T;
    im.depth = p.depth;
    im.item0 = p.item0;
    char *data = ws + L.data_off;
    im.mbuf[0] = data + p.m0;
    im.mbuf[1] = data + p.m1;
    im.mpitch = p.mpitch;
    im.bp = (uint8_t *)(data + p.bp);
    im.flags = (int *)(ws + p.flags);
    im.best = (unsigned long long *)(ws + p.best);
    im.done = (int *)(ws + p.done);
    im.x_out = p.io.x_out;
    im.d_out = p.io.d_out;
    im.score_out = p.io.score_out;
    im.win = p.io.d_window;
    im.kind = p.kind;
    im.moff = p.moff;
    im.enable = p.enable;
    im.mask1 = p.mask1;
    im.mask_x = p.mask_x;
    im.mask_end = p.mask_end;
    if (p.kind == 1) {
        im.ftiles = p.ftiles;
        im.hpitch = p.hpitch;
        im.h256 = (uint16_t *)(data + p.h256);
        im.fflags = (int *)(ws + p.fflags);
    } else if (p.kind == 2) {
        im.ftiles = p.ftiles;
        im.hwpitch = p.hpitch;
        im.hw = data + p.h256;
        im.fflags = (int *)(ws + p.fflags);
    }
    return im;
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

template <typename In, typename Acc>
int launch_kernel_wide(const LaunchArgs &args, int max_n, cudaStream_t stream) {
    using P = WideEngine<In, Acc, long long>;
    const size_t smem = P::smem_bytes(max_n, args.wpad, args.use_table != 0);
    auto kern = engine_kernel_wide<In, Acc, long long>;
    int st = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem),
                         "cudaFuncSetAttribute");
    if (st) return st;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWThreads, smem);
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)num_sms() * per_sm;
    if (grid > args.items) grid = args.items;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kWThreads, smem, stream>>>(args);
    return launched("engine_kernel_wide");
}

template <typename Key>
int launch_kernel_u8(const LaunchArgs &args, bool multi, cudaStream_t stream) {
    const size_t smem = u8_smem_bytes<Key>();
    auto kern = multi ? engine_kernel_u8<Key, true> : engine_kernel_u8<Key, false>;
    int st = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem),
                         "cudaFuncSetAttribute");
    if (st) return st;
    long long grid = num_sms();
    if (grid > args.items) grid = args.items;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kWsThreads, smem, stream>>>(args);
    return launched("engine_kernel_u8");
}

// `multi`: the run holds items of more than one tile width.
int dispatch(int dtype, int max_h, const LaunchArgs &args, int max_n, bool multi,
             cudaStream_t stream) {
    switch (dtype) {
        case FHTDP_U8:
            // 32-bit keys: values below 2^22, and dead keys (negative) that
            // take on at most 512 * (255 h + k) over the bands stay negative.
            if (256LL * max_h < (1LL << 22)) return launch_kernel_u8<int32_t>(args, multi, stream);
            return launch_kernel_u8<long long>(args, multi, stream);
        case FHTDP_I32:
            return launch_kernel_wide<int32_t, int32_t>(args, max_n, stream);
        default:
            return launch_kernel_wide<float, float>(args, max_n, stream);
    }
}

// Test hook state (per host thread), consumed by the next run.
thread_local int g_inject_band = -1, g_inject_tile = -1;
thread_local long long g_inject_wait = 0;

void consume_injection(LaunchArgs *args) {
    if (g_inject_band >= 0) {
        args->skip_band = g_inject_band;
        args->skip_tile = g_inject_tile;
        args->wait_cycles = g_inject_wait;
    }
    g_inject_band = g_inject_tile = -1;
    g_inject_wait = 0;
}

LaunchArgs base_args(const RunLayout &L, char *ws, int count) {
    LaunchArgs args{};
    args.count = count;
    args.items = L.items;
    args.ctl = (Ctl *)ws;
    args.wait_cycles = 4000000000LL;   // about two seconds at GB300 clocks
    args.skip_band = -1;
    args.skip_tile = -1;
    args.wpad = kWPad;
    consume_injection(&args);
    return args;
}

int run_fallback(const void *img, int dtype, int pitch, const Shape &s, int B, int32_t *x_out,
                 int32_t *d_out, void *score_out, void *ws, cudaStream_t stream) {
    // 256-row bands: the standalone FHT (two levels per pass), the in-place
    // DP with per-column window maxima and the read-back from a grid-wide
    // argmax.
    int st = cuda_status(cudaMemsetAsync(ws, 0, sizeof(Ctl), stream), "cudaMemsetAsync");
    if (st) return st;
    size_t hough = (size_t)s.k * 2 * s.n * s.W;
    char *base = (char *)ws + 256;
    // The argmax key sits in the cleared control block, after its fields.
    unsigned long long *key = (unsigned long long *)((char *)ws + 128);
    static_assert(sizeof(Ctl) >= 136, "control block holds the argmax key");
    if (dtype == FHTDP_F32) {
        float *H = (float *)base, *tmp = H + hough;
        st = launch_fht_stages<float, float>((const float *)img, pitch, s, H, tmp, stream);
        if (!st) st = launch_dp_inplace<float>(H, s, B, stream);
        if (!st)
            st = launch_backtrack_key<float>(H, s, B, key, x_out, d_out, (float *)score_out,
                                             stream);
        return st;
    }
    int32_t *H = (int32_t *)base, *tmp = H + hough;
    if (dtype == FHTDP_U8)
        st = launch_fht_stages<uint8_t, int32_t>((const uint8_t *)img, pitch, s, H, tmp, stream);
    else
        st = launch_fht_stages<int32_t, int32_t>((const int32_t *)img, pitch, s, H, tmp, stream);
    if (!st) st = launch_dp_inplace<int32_t>(H, s, B, stream);
    if (!st)
        st = launch_backtrack_key<int32_t>(H, s, B, key, x_out, d_out, (int32_t *)score_out,
                                           stream);
    return st;
}

ImgPlan single_plan(int dtype, const void *img, int pitch, const Shape &s, int B,
                    int32_t *x_out, int32_t *d_out, void *score_out) {
    ImgPlan p{};
    p.T = default_tile(dtype, s.n);
    p.depth = 3;
    p.io.img = img;
    p.io.h = s.h;
    p.io.w = s.w;
    p.io.pitch = pitch;
    p.io.k = s.k;
    p.io.B = B;
    p.io.x_out = x_out;
    p.io.d_out = d_out;
    p.io.score_out = score_out;
    p.s = s;
    p.B = B < 2 * s.n - 2 ? B : 2 * s.n - 2;   // wider windows change nothing
    if (fused_256(dtype, s, p.B, img, pitch)) {
        p.kind = 1;
        p.T = kTile256;
    } else if (dtype != FHTDP_U8 && s.n <= kMaxBandFused) {
        p.kind = 2;   // FHT items and narrow DP items
        p.T = kWTileD;
    }
    return p;
}

}  // namespace

// Streams over which a batch spreads its images with 256-row bands.
constexpr int kSideLanes = 4;

// The host-side plan of a batch.
struct BatchPlan {
    int dtype;
    std::vector<ImgPlan> imgs;      // images of the fused launch
    std::vector<ImgPlan> separate;  // 256-row bands: run with the standalone kernels
    size_t separate_off = 0;        // their scratch: `lanes` slices of sep_bytes
    size_t sep_bytes = 0;
    int lanes = 0;                  // streams the separate images are spread over
    std::vector<cudaStream_t> side; // one non-blocking stream per lane
    std::vector<cudaEvent_t> ev;    // fork + one join per lane
    RunLayout L;
    std::vector<ImgDesc> staging;   // image table as uploaded
    std::vector<Item> order;        // work queue as uploaded
    void *bound_ws = nullptr;
    long long target = 0;           // queue width (tiles per band level or step)
    int mode = 0;                   // queue schedule, see queue_order
    bool use_table = false;         // bend-angle windows (fhtdp_batch_angle)
    WindowTable tab{};
    size_t reserve = 0;             // bytes of the fused part for any tile-width choice
    size_t ws_total = 0;            // workspace bytes (the reserve and the side lanes)
    ~BatchPlan() {
        for (cudaStream_t st : side) cudaStreamDestroy(st);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

// Queue orders of a batch.  Both put every item after the band+1 tiles it
// waits for, so the queue cannot deadlock, and both bound the images in
// flight, whose window-maximum buffers should stay in L2.
//
// Items of a band level of an image, in tiles of 128 x 128 work (a 256-row
// band level also holds the half-band FHT items of the band above).
long long level_weight(const ImgPlan &p) {
    if (p.kind == 1) return p.tiles + 2LL * p.ftiles;
    if (p.kind == 2) return std::max(1LL, (long long)((p.tiles + 3) / 4 + (p.ftiles + 1) / 2));
    return p.tiles;
}

// The items of band level lv of one image.  256-row bands: the half-band
// FHT items of band k-1 open level 0, and each level lv also holds those of
// the band above (k-2-lv) before its DP items, so that the halves are
// ready one level ahead.
void push_level(std::vector<Item> &order, const ImgPlan &p, int i, int lv) {
    const int b = p.s.k - 1 - lv;
    if (p.kind == 1 || p.kind == 2) {
        // FHT items of a band: both halves' tiles (256-row bands) or its tiles
        // (256-row bands: the halves of band b-1 in a block before the DP items
        // of band b; their DP items wait mostly for those of band b+1)
        const long long F = p.kind == 1 ? 2LL * p.ftiles : p.ftiles;
        const WideLevels wl{p.s.k, F, p.tiles, p.kind == 1 ? 1 : kWAhead, p.kind != 1};
        const long long len = wl.start(lv + 1) - wl.start(lv);
        for (long long off = 0; off < len; ++off) {
            int dp, band, tile;
            wl.at(lv, off, &dp, &band, &tile);
            int kind;
            if (p.kind == 2) {
                kind = dp ? kItemWideDp : kItemWideFht;
            } else if (dp) {
                kind = kItemDp256;
            } else {
                kind = kItemHalf0 + tile / p.ftiles;
                tile %= p.ftiles;
            }
            order.push_back(Item{i, band, tile, kind << 19});
        }
        return;
    }
    for (int t = 0; t < p.tiles; ++t) order.push_back(Item{i, b, t, kItemBand << 19});
}

// Groups: images are taken in groups whose band levels hold about `target`
// tiles each; inside a group the items go band level by band level (the last
// band of every image first), image by image, tile by tile, so the band
// chains of a whole group advance together.  The batch is split into
// round(total / target) groups of about equal width, so that no narrow
// remainder group runs its band chain alone at the end.
std::vector<Item> queue_grouped(const std::vector<ImgPlan> &imgs, long long target) {
    std::vector<Item> order;
    long long total = 0;
    for (const ImgPlan &p : imgs) total += level_weight(p);
    const long long groups = std::max(1LL, (total + target / 2) / std::max(1LL, target));
    size_t first = 0;
    long long done = 0;
    for (long long g = 1; first < imgs.size(); ++g) {
        const long long goal = total * g / groups;
        size_t last = first;
        while (last < imgs.size() &&
               (last == first || done + level_weight(imgs[last]) / 2 < goal)) {
            done += level_weight(imgs[last]);
            ++last;
        }
        int levels = 0;
        for (size_t i = first; i < last; ++i) levels = std::max(levels, imgs[i].s.k);
        for (int lv = 0; lv < levels; ++lv)
            for (size_t i = first; i < last; ++i)
                if (lv < imgs[i].s.k) push_level(order, imgs[i], (int)i, lv);
        first = last;
    }
    return order;
}

// Band chains: an active set of images advances one band level per step,
// each step holding every active image's next level, image by image, tile
// by tile.  Images join the set, the longest chains (most bands) first,
// whenever its width (tiles per step) drops below `target`, so that steps
// keep about the same width while images of different heights finish at
// different times, and the longest chains start with the batch.
// With `mixed`, the images of 256-row bands (at most 16 bands, but heavy DP
// items that wait for nine producer tiles each) are spread evenly through
// the join order of the others (which stays longest chain first), so that
// they do not all end up in the last steps, waiting on one another.
// With `slow256`, images of 256-row bands advance one level every second
// step: a DP item of such a band waits for nine DP items of the band below,
// which are then two steps ahead of it in the queue.
std::vector<Item> queue_chains(const std::vector<ImgPlan> &imgs, long long target,
                               bool mixed = false, bool slow256 = false) {
    // the longest band chains first, so that they start with the batch
    std::vector<int> by_k(imgs.size());
    for (size_t i = 0; i < imgs.size(); ++i) by_k[i] = (int)i;
    std::stable_sort(by_k.begin(), by_k.end(),
                     [&](int a, int b) { return imgs[a].s.k > imgs[b].s.k; });
    if (mixed) {
        // rank of each image within its group (256-row bands or the others),
        // as a fraction of the group's size
        std::vector<double> key(imgs.size());
        for (int heavy = 0; heavy < 2; ++heavy) {
            int count = 0, rank = 0;
            for (int i : by_k) count += (imgs[i].kind == 1) == (heavy == 1);
            for (int i : by_k)
                if ((imgs[i].kind == 1) == (heavy == 1)) key[i] = (rank++ + 0.5) / count;
        }
        std::stable_sort(by_k.begin(), by_k.end(), [&](int a, int b) { return key[a] < key[b]; });
    }
    std::vector<Item> order;
    struct Active {
        int image, level;
        long long step0;   // the step it joined
    };
    std::vector<Active> active;
    long long step = 0;
    size_t next = 0;
    long long width = 0;
    target = std::max(1LL, target);
    while (next < imgs.size() || !active.empty()) {
        while (next < imgs.size() && (active.empty() || width < target)) {
            active.push_back(Active{by_k[next], 0, step});
            width += level_weight(imgs[by_k[next]]);
            ++next;
        }
        std::vector<Active> still;
        for (Active &a : active) {
            const ImgPlan &p = imgs[a.image];
            if (slow256 && p.kind == 1 && (step - a.step0) % 2 != 0) {
                still.push_back(a);
                continue;
            }
            push_level(order, p, a.image, a.level);
            if (++a.level < p.s.k)
                still.push_back(a);
            else
                width -= level_weight(p);
        }
        active.swap(still);
        ++step;
    }
    return order;
}

// The queue order of a schedule: 0 groups of images advancing together
// (queue_grouped); band chains joining as others finish, longest first
// (queue_chains): 1 as they are, 2 with the images of 256-row bands spread
// through the join order, 3 with 256-row bands advancing every second step,
// 4 both.
constexpr int kSchedules = 5;
std::vector<Item> queue_order(const std::vector<ImgPlan> &imgs, long long target, int mode) {
    return mode ? queue_chains(imgs, target, mode == 2 || mode == 4, mode >= 3)
                : queue_grouped(imgs, target);
}

size_t engine_workspace_bytes(int dtype, const Shape &s, int B) {
    const size_t standalone = 256 + 2 * (size_t)s.k * 2 * s.n * s.W * 4;
    if (s.n > kMaxBandFused) {
        // Either path may run, depending on the image's alignment.
        const int Bc = B < 2 * s.n - 2 ? B : 2 * s.n - 2;
        if (dtype != FHTDP_U8 || Bc > 127) return standalone;
        std::vector<ImgPlan> one{single_plan(dtype, nullptr, 16, s, B, nullptr, nullptr, nullptr)};
        return std::max(standalone, plan_layout(one, false).total);
    }
    std::vector<ImgPlan> one{single_plan(dtype, nullptr, s.w, s, B, nullptr, nullptr, nullptr)};
    return plan_layout(one, false).total;
}

// The point of Subproblems 2-3 on an image's plan: the states of band j whose
// start is not xp die, or for j = k those of band k-1 whose end is not xp.
void set_point(ImgPlan &p, int j, int xp) {
    p.mask1 = (j < p.s.k ? j : p.s.k - 1) + 1;
    p.mask_x = xp;
    p.mask_end = j == p.s.k ? 1 : 0;
}

// The fused engine masks the point's band in V after forming it, which band
// 0 never stores: points on borders 1..k of uint8 images with at least two
// bands of at most 128 rows.
bool engine_takes_point(int dtype, const Shape &s, int j) {
    return dtype == FHTDP_U8 && s.n <= kMaxBandFused && s.k >= 2 && j >= 1;
}

int engine_detect(const void *img, int dtype, int pitch, const Shape &s, int B, int32_t *x_out,
                  int32_t *d_out, void *score_out, void *ws, size_t ws_bytes, cudaStream_t stream,
                  const PointMask *pm) {
    (void)ws_bytes;
    std::vector<ImgPlan> one{single_plan(dtype, img, pitch, s, B, x_out, d_out, score_out)};
    if (pm) {
        if (!engine_takes_point(dtype, s, pm->j) || one[0].kind != 0)
            return set_error(FHTDP_EINVAL, "the fused engine takes points on uint8 images only");
        set_point(one[0], pm->j, pm->xp);
    }
    if (s.n > kMaxBandFused && one[0].kind != 1)
        return run_fallback(img, dtype, pitch, s, B, x_out, d_out, score_out, ws, stream);
    RunLayout L = plan_layout(one, false);
    char *base = (char *)ws;
    int st = cuda_status(cudaMemsetAsync(base, 0, L.zero_bytes, stream), "cudaMemsetAsync");
    if (st) return st;
    LaunchArgs args = base_args(L, base, 1);
    args.one = make_desc(one[0], L, base, dtype);
    if (one[0].kind == 1 && (!args.one.use_tma || !args.one.use_mtma))
        return set_error(FHTDP_ECUDA, "tensor maps of a 256-row-band image could not be encoded");
    args.many = nullptr;
    args.order = nullptr;
    return dispatch(dtype, L.max_h, args, L.max_n, L.multi_tile, stream);
}

// The window table's cover in the DP items: the shortest window that no end
// of the range clips (else the shortest of all), made odd, is 2 B0 + 1; every
// window at least as long is covered by pieces of that length, every shorter
// one is clipped.  The centred maxima read V up to 2 B0 + 16 rows beyond the
// range, so the dead pad holds that many rows (even, for the copies' 128-byte
// alignment).
void set_table(LaunchArgs &args, const WindowTable &t) {
    const int n = t.n, D = 2 * n - 1;
    int L0 = D, L0c = D;
    bool any = false;
    for (int i = 0; i < D; ++i) {
        const int len = t.hi[i] - t.lo[i] + 1;
        L0c = std::min(L0c, len);
        if (t.lo[i] > -(n - 1) && t.hi[i] < n - 1) {
            L0 = any ? std::min(L0, len) : len;
            any = true;
        }
    }
    if (!any) L0 = L0c;
    if (L0 < 1) L0 = 1;
    const int Lp = L0 % 2 ? L0 : L0 - 1;
    args.use_table = 1;
    args.tab = t;
    args.B0 = (Lp - 1) / 2;
    args.wpad = std::max(kWPad, (2 * args.B0 + 16 + 1) & ~1);
}

// One int32 / float image with the bend-angle windows of table t (bands of 2
// to 128 rows): the persistent engine with window-table DP items.
int engine_detect_table(const void *img, int dtype, int pitch, const Shape &s,
                        const WindowTable &t, int32_t *x_out, int32_t *d_out, void *score_out,
                        void *ws, cudaStream_t stream) {
    if (dtype == FHTDP_U8 || s.n < 2 || s.n > kMaxBandFused || t.n != s.n)
        return set_error(FHTDP_EINVAL, "window-table engine: int32 / float, bands of 2..128 rows");
    std::vector<ImgPlan> one{single_plan(dtype, img, pitch, s, 2 * s.n - 2, x_out, d_out,
                                         score_out)};
    RunLayout L = plan_layout(one, false);
    char *base = (char *)ws;
    int st = cuda_status(cudaMemsetAsync(base, 0, L.zero_bytes, stream), "cudaMemsetAsync");
    if (st) return st;
    LaunchArgs args = base_args(L, base, 1);
    args.one = make_desc(one[0], L, base, dtype);
    args.many = nullptr;
    args.order = nullptr;
    set_table(args, t);
    return dispatch(dtype, L.max_h, args, L.max_n, false, stream);
}

int engine_status(const void *ws, cudaStream_t stream) {
    int status = 0;
    int st = cuda_status(cudaMemcpyAsync(&status, (const char *)ws + offsetof(Ctl, status),
                                         sizeof(int), cudaMemcpyDeviceToHost, stream),
                         "cudaMemcpyAsync");
    if (st) return st;
    st = cuda_status(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    if (st) return st;
    if (status != FHTDP_OK) return set_error(status, "a device-side wait gave up");
    return FHTDP_OK;
}

int batch_create(const fhtdp_image *images, int count, int dtype, BatchPlan **out) {
    if (count < 1 || !images) return set_error(FHTDP_EINVAL, "empty batch");
    BatchPlan *plan = new (std::nothrow) BatchPlan();
    if (!plan) return set_error(FHTDP_EINVAL, "out of host memory");
    plan->dtype = dtype;
    for (int i = 0; i < count; ++i) {
        const fhtdp_image &io = images[i];
        Shape s;
        if (!make_shape(io.h, io.w, io.k, &s) || io.pitch < io.w || io.B < 0 || !io.img ||
            !io.x_out || !io.d_out || !io.score_out) {
            delete plan;
            return set_error(FHTDP_EINVAL,
                             "image %d: invalid (h=%d w=%d pitch=%d k=%d B=%d or null pointer)",
                             i, io.h, io.w, io.pitch, io.k, io.B);
        }
        ImgPlan p = single_plan(dtype, io.img, io.pitch, s, io.B, io.x_out, io.d_out, io.score_out);
        p.io.d_window = io.d_window;
        if (io.d_window && s.n > kMaxBandFused) {
            delete plan;
            return set_error(FHTDP_EINVAL,
                             "image %d: displacement windows need bands of at most %d rows", i,
                             kMaxBandFused);
        }
        if (s.n > kMaxBandFused && p.kind != 1)
            plan->separate.push_back(p);
        else
            plan->imgs.push_back(p);
    }
    plan->L = plan_layout(plan->imgs, true);
    {
        std::vector<ImgPlan> any = plan->imgs;
        plan->reserve = plan_layout(any, true, true, dtype).total;
    }
    // Scratch of the standalone path: up to kSideLanes lanes, each a stream
    // that runs its images one after the other on its own slice.
    size_t sep = 0;
    for (auto &p : plan->separate) sep = std::max(sep, engine_workspace_bytes(dtype, p.s, p.io.B));
    plan->sep_bytes = align_up(sep, 256);
    plan->lanes = (int)std::min<size_t>(kSideLanes, plan->separate.size());
    plan->separate_off = align_up(plan->reserve, 256);
    plan->ws_total = sep ? plan->separate_off + plan->sep_bytes * plan->lanes : plan->reserve;
    for (int l = 0; l < plan->lanes; ++l) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            delete plan;
            return cuda_status(cudaGetLastError(), "cudaStreamCreateWithFlags");
        }
        plan->side.push_back(st);
    }
    for (int l = 0; plan->lanes && l <= plan->lanes; ++l) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            delete plan;
            return cuda_status(cudaGetLastError(), "cudaEventCreateWithFlags");
        }
        plan->ev.push_back(e);
    }
    plan->target = num_sms();
    plan->order = queue_order(plan->imgs, plan->target, plan->mode);
    *out = plan;
    return FHTDP_OK;
}

// Each queue entry carries its image's band height and TMA flag.
void set_nflags(BatchPlan *plan) {
    for (Item &it : plan->order)
        it.nflags = (it.nflags & (3 << 19)) | plan->imgs[it.image].s.n |
                    (plan->staging[it.image].use_tma ? 1 << 16 : 0) |
                    (tile_code(plan->imgs[it.image].T) << 17);
}

size_t batch_workspace_bytes(const BatchPlan *plan) { return plan ? plan->ws_total : 0; }

long long batch_items(const BatchPlan *plan) { return plan ? plan->L.items : 0; }

// The image table and the queue of the plan's current layout into `ws`.
int upload_tables(BatchPlan *plan, void *ws, cudaStream_t stream) {
    plan->staging.clear();
    for (auto &p : plan->imgs) {
        plan->staging.push_back(make_desc(p, plan->L, (char *)ws, plan->dtype));
        const ImgDesc &im = plan->staging.back();
        if (p.kind == 1 && (!im.use_tma || !im.use_mtma))
            return set_error(FHTDP_ECUDA,
                             "tensor maps of a 256-row-band image could not be encoded");
    }
    set_nflags(plan);
    int st = cuda_status(cudaMemcpyAsync((char *)ws + plan->L.table_off, plan->staging.data(),
                                         sizeof(ImgDesc) * plan->staging.size(),
                                         cudaMemcpyHostToDevice, stream),
                         "cudaMemcpyAsync");
    if (st) return st;
    return cuda_status(cudaMemcpyAsync((char *)ws + plan->L.order_off, plan->order.data(),
                                       sizeof(Item) * plan->order.size(),
                                       cudaMemcpyHostToDevice, stream),
                       "cudaMemcpyAsync");
}

int batch_upload(BatchPlan *plan, void *ws, size_t ws_bytes, cudaStream_t stream) {
    if (!plan || !ws) return set_error(FHTDP_EINVAL, "null plan or workspace");
    if (ws_bytes < plan->ws_total)
        return set_error(FHTDP_EWORKSPACE, "batch workspace needs %zu bytes, got %zu",
                         plan->ws_total, ws_bytes);
    plan->bound_ws = ws;
    return upload_tables(plan, ws, stream);
}

int batch_run(const BatchPlan *plan, void *ws, cudaStream_t stream) {
    if (!plan || !ws) return set_error(FHTDP_EINVAL, "null plan or workspace");
    if (ws != plan->bound_ws)
        return set_error(FHTDP_EINVAL, "workspace differs from the one given to fhtdp_batch_upload");
    char *base = (char *)ws;
    int st = cuda_status(cudaMemsetAsync(base, 0, plan->L.zero_bytes, stream), "cudaMemsetAsync");
    if (st) return st;
    // Images with 256-row bands: the standalone kernels, spread over the
    // plan's lanes (forked from and joined back into `stream` by events, so
    // the run stays one stream-ordered operation for the caller).
    if (plan->lanes) {
        st = cuda_status(cudaEventRecord(plan->ev[0], stream), "cudaEventRecord");
        for (int l = 0; l < plan->lanes && !st; ++l)
            st = cuda_status(cudaStreamWaitEvent(plan->side[l], plan->ev[0], 0),
                             "cudaStreamWaitEvent");
        for (size_t i = 0; i < plan->separate.size() && !st; ++i) {
            const ImgPlan &p = plan->separate[i];
            const int l = (int)(i % plan->lanes);
            st = run_fallback(p.io.img, plan->dtype, p.io.pitch, p.s, p.io.B, p.io.x_out,
                              p.io.d_out, p.io.score_out,
                              base + plan->separate_off + plan->sep_bytes * l, plan->side[l]);
        }
    }
    if (!plan->imgs.empty() && !st) {
        LaunchArgs args = base_args(plan->L, base, (int)plan->imgs.size());
        args.many = (const ImgDesc *)(base + plan->L.table_off);
        args.order = (const Item *)(base + plan->L.order_off);
        if (plan->use_table) set_table(args, plan->tab);
        st = dispatch(plan->dtype, plan->L.max_h, args, plan->L.max_n, plan->L.multi_tile, stream);
    }
    // Join the lanes back (also after an error, so that `stream` never runs
    // ahead of work it forked).
    for (int l = 0; l < plan->lanes; ++l) {
        int js = cuda_status(cudaEventRecord(plan->ev[1 + l], plan->side[l]), "cudaEventRecord");
        if (!js)
            js = cuda_status(cudaStreamWaitEvent(stream, plan->ev[1 + l], 0),
                             "cudaStreamWaitEvent");
        if (!st) st = js;
    }
    return st ? st : FHTDP_OK;
}

// Tunes the bound batch by timing runs (synchronising `stream` after every
// candidate) and keeps the fastest of each choice in turn:
//   1. the queue schedule (groups or band chains) and its width, from half a
//      wave to the whole batch at once (wider steps wait less for
//      dependencies but keep more window-maximum buffers in flight in L2);
//   2. for each band height of the uint8 images, the column tile width of
//      its items (128 or 256 columns where shared memory allows) and the
//      number of FHT levels done in registers before the shared-memory merges
//      (2 or 3), applied to every image of that height;
//   3. the schedule again, for the tile widths chosen.
// Leaves the workspace with the chosen layout and queue uploaded.
int batch_autotune(BatchPlan *plan, void *ws, int reps, cudaStream_t stream, long long *chosen) {
    if (!plan || !ws) return set_error(FHTDP_EINVAL, "null plan or workspace");
    if (ws != plan->bound_ws)
        return set_error(FHTDP_EINVAL, "workspace differs from the one given to fhtdp_batch_upload");
    if (reps < 1) reps = 1;
    if (plan->imgs.empty()) {
        if (chosen) *chosen = plan->target;
        return FHTDP_OK;
    }
    const long long sms = num_sms();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = cuda_status(cudaEventCreate(&e0), "cudaEventCreate");
    if (!st) st = cuda_status(cudaEventCreate(&e1), "cudaEventCreate");
    // Runs of the current layout and queue: warm-up, then `reps` timed; the
    // first candidate raises `reps` so that each candidate is timed over
    // about 8 ms (short batches are otherwise within the timing noise).
    bool sized = false;
    auto time_runs = [&](float *ms) -> int {
        int r = batch_run(plan, ws, stream);
        if (!r) r = cuda_status(cudaEventRecord(e0, stream), "cudaEventRecord");
        for (int i = 0; i < reps && !r; ++i) r = batch_run(plan, ws, stream);
        if (!r) r = cuda_status(cudaEventRecord(e1, stream), "cudaEventRecord");
        if (!r) r = cuda_status(cudaEventSynchronize(e1), "cudaEventSynchronize");
        if (!r) r = cuda_status(cudaEventElapsedTime(ms, e0, e1), "cudaEventElapsedTime");
        if (!r) *ms /= reps;
        if (!r && !sized) {
            sized = true;
            if (*ms > 0.0f) reps = std::max(reps, std::min(64, (int)(8.0f / *ms)));
        }
        return r;
    };
    // Lays the plan out again (tile widths may have changed) and uploads it.
    auto apply = [&](long long t, int mode) -> int {
        plan->L = plan_layout(plan->imgs, true);
        if (plan->L.total > plan->reserve)
            return set_error(FHTDP_EWORKSPACE, "tuned layout exceeds the reserved workspace");
        plan->order = queue_order(plan->imgs, t, mode);
        return upload_tables(plan, ws, stream);
    };
    float best_ms = -1.0f;
    auto tune_schedule = [&]() -> int {
        long long total = 0;
        for (const ImgPlan &p : plan->imgs) total += level_weight(p);
        std::vector<long long> cands;
        const long long widths[] = {sms / 2, 3 * sms / 4, sms, 3 * sms / 2, 2 * sms, 3 * sms,
                                    4 * sms, 6 * sms, total};
        for (long long t : widths) {
            if (t < 1) continue;
            t = std::min(t, total);   // every width of at least the batch gives one order
            if (std::find(cands.begin(), cands.end(), t) == cands.end()) cands.push_back(t);
        }
        long long bt = plan->target;
        int bm = plan->mode;
        float bms = -1.0f;
        int r = 0;
        for (size_t c = 0; c < kSchedules * cands.size() && !r; ++c) {
            const int mode = (int)(c / cands.size());
            const long long t = cands[c % cands.size()];
            r = apply(t, mode);
            float ms = 0.0f;
            if (!r) r = time_runs(&ms);
            if (!r && (bms < 0.0f || ms < bms)) {
                bms = ms;
                bt = t;
                bm = mode;
            }
        }
        plan->target = bt;
        plan->mode = bm;
        best_ms = bms;
        return r;
    };
    if (!st) st = tune_schedule();
    if (!st && plan->dtype == FHTDP_U8) {
        std::vector<int> heights;
        for (const ImgPlan &p : plan->imgs)
            if (std::find(heights.begin(), heights.end(), p.s.n) == heights.end())
                heights.push_back(p.s.n);
        for (size_t hi = 0; hi < heights.size() && !st; ++hi) {
            const int n = heights[hi];
            if (n < 4) continue;   // no register levels to choose, one tile width
            ImgPlan *first = nullptr;
            for (ImgPlan &p : plan->imgs)
                if (p.s.n == n) {
                    first = &p;
                    break;
                }
            const int T0 = first->T, D0 = first->depth;
            int bT = T0, bD = D0;
            const int Ts[2] = {kTile, 2 * kTile};
            for (int ti = 0; ti < 2 && !st; ++ti)
                for (int depth = 2; depth <= 3 && !st; ++depth) {
                    const int T = first->kind == 1 ? T0 : Ts[ti];
                    if (ti == 1 && first->kind == 1) continue;
                    if (!tile_choice(plan->dtype, *first, T)) continue;
                    if (depth == 3 && n < 8) continue;
                    if (T == T0 && depth == D0) continue;   // timed already
                    for (ImgPlan &p : plan->imgs)
                        if (p.s.n == n) {
                            p.T = T;
                            p.depth = depth;
                        }
                    st = apply(plan->target, plan->mode);
                    float ms = 0.0f;
                    if (!st) st = time_runs(&ms);
                    if (!st && ms < best_ms) {
                        best_ms = ms;
                        bT = T;
                        bD = depth;
                    }
                }
            for (ImgPlan &p : plan->imgs)
                if (p.s.n == n) {
                    p.T = bT;
                    p.depth = bD;
                }
        }
        if (!st) st = tune_schedule();
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // Whatever happened, leave the plan and the workspace with one layout.
    const int us = apply(plan->target, plan->mode);
    if (!st) st = us;
    if (!st) st = cuda_status(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    if (chosen) *chosen = plan->target;
    return st;
}

// Sets the tile width and register FHT depth of the plan's images of band
// height n and uploads the new layout and queue into its bound workspace.
int batch_configure(BatchPlan *plan, void *ws, int n, int tile, int depth, cudaStream_t stream) {
    if (!plan || !ws) return set_error(FHTDP_EINVAL, "null plan or workspace");
    if (ws != plan->bound_ws)
        return set_error(FHTDP_EINVAL, "workspace differs from the one given to fhtdp_batch_upload");
    bool any = false;
    for (const ImgPlan &p : plan->imgs) {
        if (p.s.n != n) continue;
        any = true;
        if (!tile_choice(plan->dtype, p, tile))
            return set_error(FHTDP_EINVAL, "tile width %d not available for band height %d",
                             tile, n);
        if (depth < 2 || depth > 3 || (depth == 3 && n < 8))
            return set_error(FHTDP_EINVAL, "register depth %d not available for band height %d",
                             depth, n);
    }
    if (!any) return set_error(FHTDP_EINVAL, "no image of band height %d in the fused launch", n);
    for (ImgPlan &p : plan->imgs)
        if (p.s.n == n) {
            p.T = tile;
            p.depth = depth;
        }
    plan->L = plan_layout(plan->imgs, true);
    plan->order = queue_order(plan->imgs, plan->target, plan->mode);
    return upload_tables(plan, ws, stream);
}

// The plan's queue schedule and width, and the tile width and register
// depth of its images of band height n (0 when it has none).
void batch_choice(const BatchPlan *plan, int n, int *mode, long long *target, int *tile,
                  int *depth) {
    if (mode) *mode = plan->mode;
    if (target) *target = plan->target;
    int T = 0, dd = 0;
    for (const ImgPlan &p : plan->imgs)
        if (p.s.n == n) {
            T = p.T;
            dd = p.depth;
            break;
        }
    if (tile) *tile = T;
    if (depth) *depth = dd;
}

// Image i of the fused launch runs only where enable[i] reads nonzero at the
// launch (set before fhtdp_batch_upload).
void batch_set_enable(BatchPlan *plan, const int32_t *enable) {
    for (size_t i = 0; i < plan->imgs.size(); ++i) plan->imgs[i].enable = enable ? enable + i : nullptr;
}

int batch_separate_count(const BatchPlan *plan) { return (int)plan->separate.size(); }

int batch_points(BatchPlan *plan, void *ws, const int32_t *points, cudaStream_t stream) {
    if (!plan || !points) return set_error(FHTDP_EINVAL, "null plan or points");
    if (ws != plan->bound_ws)
        return set_error(FHTDP_EINVAL, "workspace differs from the one given to fhtdp_batch_upload");
    if (!plan->separate.empty())
        return set_error(FHTDP_EINVAL, "points: the batch has images outside the fused engine");
    // The images in the caller's order are the plan's images (none separate).
    for (size_t i = 0; i < plan->imgs.size(); ++i) {
        const int j = points[2 * i], xp = points[2 * i + 1];
        const ImgPlan &p = plan->imgs[i];
        if (j < 0) continue;
        if (j > p.s.k || xp < 0 || xp >= p.s.w || p.kind != 0 ||
            !engine_takes_point(plan->dtype, p.s, j))
            return set_error(FHTDP_EINVAL,
                             "point %zu: border 1..k, column 0..w-1, uint8, 2+ bands of <= 128 rows",
                             i);
    }
    for (size_t i = 0; i < plan->imgs.size(); ++i) {
        ImgPlan &p = plan->imgs[i];
        p.mask1 = 0;
        if (points[2 * i] >= 0) set_point(p, points[2 * i], points[2 * i + 1]);
    }
    return upload_tables(plan, ws, stream);
}

int batch_angle(BatchPlan *plan, double gamma) {
    if (!plan) return set_error(FHTDP_EINVAL, "null plan");
    if (plan->dtype == FHTDP_U8 || !plan->separate.empty() || plan->imgs.empty())
        return set_error(FHTDP_EINVAL,
                         "bend-angle batches: int32 / float images with bands of 2..128 rows");
    const int n = plan->imgs[0].s.n;
    for (const ImgPlan &p : plan->imgs)
        if (p.s.n != n || p.kind != 2 || n < 2)
            return set_error(FHTDP_EINVAL,
                             "bend-angle batches: one band height of 2..128 rows for all images");
    WindowTable t;
    if (!make_angle_table(n, gamma, &t)) return set_error(FHTDP_EINVAL, "gamma must be >= 0");
    plan->tab = t;
    plan->use_table = true;
    return FHTDP_OK;
}

void batch_destroy(BatchPlan *plan) { delete plan; }

void debug_inject(int band, int tile, long long wait_cycles) {
    g_inject_band = band;
    g_inject_tile = tile;
    g_inject_wait = wait_cycles > 0 ? wait_cycles : 1;
}

}  // namespace fhtdp
