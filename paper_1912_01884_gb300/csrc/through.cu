// Subproblems 2-3 (Sec. 2.2-2.3) on one image: the extreme polyline through a
// given point P on a band border.  Host side only: the sequence of launches.
//
// The paper builds the part below P by the DP over bands j..k-1 and the part
// above P by the same DP on bands 0..j-1 flipped about Ox.  Here one DP runs
// over all bands and marks every state of P's band whose vertex on P's
// border is not xp dead, so the optimum over V_0 is the best polyline through
// P with the bend limit at every vertex, P included, and the usual read-back
// (Eq. 5) returns it.
#include "common.cuh"

namespace fhtdp {

namespace {
constexpr size_t kThroughHead = 256;   // the argmax key, cleared by every call

size_t round_up256(size_t v) { return (v + 255) & ~(size_t)255; }
}  // namespace

// [head][Hough/V k*2n*W 4-byte][FHT scratch, same]
size_t through_workspace_bytes(const Shape &s) {
    return kThroughHead + 2 * round_up256((size_t)s.k * 2 * s.n * s.W * 4);
}

int detect_through(const void *img, int dtype, int pitch, const Shape &s, int B,
                   const PointMask &pm, int32_t *x_out, int32_t *d_out, int32_t *score_out,
                   void *ws, cudaStream_t stream) {
    char *base = (char *)ws;
    unsigned long long *key = (unsigned long long *)base;
    int32_t *H = (int32_t *)(base + kThroughHead);
    int32_t *tmp = H + round_up256((size_t)s.k * 2 * s.n * s.W * 4) / 4;
    int st = cuda_status(cudaMemsetAsync(base, 0, kThroughHead, stream), "cudaMemsetAsync");
    if (st) return st;
    st = dtype == FHTDP_U8
             ? launch_fht_stages<uint8_t, int32_t>((const uint8_t *)img, pitch, s, H, tmp, stream)
             : launch_fht_stages<int32_t, int32_t>((const int32_t *)img, pitch, s, H, tmp, stream);
    if (!st) st = launch_dp_inplace<int32_t>(H, s, B, stream, &pm);
    if (!st) st = launch_backtrack_key<int32_t>(H, s, B, key, x_out, d_out, score_out, stream);
    return st;
}

}  // namespace fhtdp
