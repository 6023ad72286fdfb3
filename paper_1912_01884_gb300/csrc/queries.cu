// Queries on the standalone kernels, host side only (the sequences of
// launches).
//
// Subproblems 2-3 (Sec. 2.2-2.3): the extreme polyline through a given point
// P on a band border.
// The paper builds the part below P by the DP over bands j..k-1 and the part
// above P by the same DP on bands 0..j-1 flipped about Ox.  Here one DP runs
// over all bands and marks every state of P's band whose vertex on P's
// border is not xp dead, so the optimum over V_0 is the best polyline through
// P with the bend limit at every vertex, P included, and the usual read-back
// (Eq. 5) returns it.
#include <type_traits>

#include "common.cuh"
#include "engine.cuh"

namespace fhtdp {

namespace {
constexpr size_t kThroughHead = 256;   // the argmax key, cleared by every call

size_t round_up256(size_t v) { return (v + 255) & ~(size_t)255; }
}  // namespace

// [head][Hough/V k*2n*W 4-byte values][FHT scratch, same]; uint8 images with
// bands of at most 128 rows run the through-point query in the fused engine,
// whose workspace is smaller for all but the narrowest images.
size_t through_workspace_bytes(const Shape &s) {
    size_t need = kThroughHead + 2 * round_up256((size_t)s.k * 2 * s.n * s.W * 4);
    if (engine_takes_point(FHTDP_U8, s)) {
        const size_t eng = engine_workspace_bytes(FHTDP_U8, s, 0);
        if (eng > need) need = eng;
    }
    return need;
}

namespace {
// The band FHTs of an image of any dtype into H (int32 for integer images,
// float for float32 ones).
template <typename Acc>
int fht_any(const void *img, int dtype, int pitch, const Shape &s, Acc *H, Acc *tmp,
            cudaStream_t stream) {
    if constexpr (std::is_same<Acc, float>::value) {
        return launch_fht_stages<float, float>((const float *)img, pitch, s, H, tmp, stream);
    } else {
        return dtype == FHTDP_U8
                   ? launch_fht_stages<uint8_t, int32_t>((const uint8_t *)img, pitch, s, H, tmp,
                                                         stream)
                   : launch_fht_stages<int32_t, int32_t>((const int32_t *)img, pitch, s, H, tmp,
                                                         stream);
    }
}

template <typename Acc>
int detect_through_t(const void *img, int dtype, int pitch, const Shape &s, int B,
                     const PointMask *pm, int32_t *x_out, int32_t *d_out, Acc *score_out,
                     void *ws, cudaStream_t stream) {
    char *base = (char *)ws;
    unsigned long long *key = (unsigned long long *)base;
    Acc *H = (Acc *)(base + kThroughHead);
    Acc *tmp = H + round_up256((size_t)s.k * 2 * s.n * s.W * 4) / 4;
    int st = cuda_status(cudaMemsetAsync(base, 0, kThroughHead, stream), "cudaMemsetAsync");
    if (st) return st;
    st = fht_any<Acc>(img, dtype, pitch, s, H, tmp, stream);
    if (!st) st = launch_dp_inplace<Acc>(H, s, B, stream, pm);
    if (!st) st = launch_backtrack_key<Acc>(H, s, B, key, x_out, d_out, score_out, stream);
    return st;
}

template <typename Acc>
int detect_two_t(const void *img, int dtype, int pitch, const Shape &s, int B, int sep,
                 int32_t *x_out, int32_t *d_out, Acc *score_out, void *ws, cudaStream_t stream) {
    char *base = (char *)ws;
    unsigned long long *key1 = (unsigned long long *)base, *key2 = key1 + 1;
    Acc *H = (Acc *)(base + kThroughHead);
    Acc *tmp = H + round_up256((size_t)s.k * 2 * s.n * s.W * 4) / 4;
    int st = cuda_status(cudaMemsetAsync(base, 0, kThroughHead, stream), "cudaMemsetAsync");
    if (st) return st;
    st = fht_any<Acc>(img, dtype, pitch, s, H, tmp, stream);
    if (!st) st = launch_dp_inplace<Acc>(H, s, B, stream);
    if (!st) st = launch_backtrack_key<Acc>(H, s, B, key1, x_out, d_out, score_out, stream);
    if (!st) st = launch_argmax_apart<Acc>(H, s, key1, sep, key2, stream);
    if (!st)
        st = launch_readback_key<Acc>(H, s, B, key2, x_out + s.k + 1, d_out + s.k, score_out + 1,
                                      stream);
    return st;
}
}  // namespace

int detect_through(const void *img, int dtype, int pitch, const Shape &s, int B,
                   const PointMask &pm, int32_t *x_out, int32_t *d_out, void *score_out,
                   void *ws, cudaStream_t stream) {
    // uint8 images with bands of at most 128 rows, P on borders 1..k: the
    // fused engine with P's band masked once its V is formed (the same DP as
    // below)
    if (engine_takes_point(dtype, s, pm.j))
        return engine_detect(img, dtype, pitch, s, B, x_out, d_out, score_out, ws,
                             through_workspace_bytes(s), stream, &pm);
    if (dtype == FHTDP_F32)
        return detect_through_t<float>(img, dtype, pitch, s, B, &pm, x_out, d_out,
                                       (float *)score_out, ws, stream);
    return detect_through_t<int32_t>(img, dtype, pitch, s, B, &pm, x_out, d_out,
                                     (int32_t *)score_out, ws, stream);
}

// Vertices anywhere in the zero-padded band width (Sec. 2.2: Hough columns
// up to w + h/k - 1).  The cyclic FHT never wraps for a link with both ends
// in [0, W), so its values are the plain sums with zeros right of the image;
// the DP and the read-back run over the vertex domain s.vw = W.
int detect_padded(const void *img, int dtype, int pitch, const Shape &s, int B, int32_t *x_out,
                  int32_t *d_out, void *score_out, void *ws, cudaStream_t stream) {
    if (dtype == FHTDP_F32)
        return detect_through_t<float>(img, dtype, pitch, s, B, nullptr, x_out, d_out,
                                       (float *)score_out, ws, stream);
    return detect_through_t<int32_t>(img, dtype, pitch, s, B, nullptr, x_out, d_out,
                                     (int32_t *)score_out, ws, stream);
}

// Two different extreme polylines (Sec. 3, Figs. 6d and 7a; the paper gives
// no rule): the optimum, then the best polyline whose top vertex lies at
// least sep columns from the optimum's, both read back from the same V.
// Workspace as for the through-point query; the second key follows the first.
int detect_two(const void *img, int dtype, int pitch, const Shape &s, int B, int sep,
               int32_t *x_out, int32_t *d_out, void *score_out, void *ws, cudaStream_t stream) {
    if (dtype == FHTDP_F32)
        return detect_two_t<float>(img, dtype, pitch, s, B, sep, x_out, d_out, (float *)score_out,
                                   ws, stream);
    return detect_two_t<int32_t>(img, dtype, pitch, s, B, sep, x_out, d_out,
                                 (int32_t *)score_out, ws, stream);
}

}  // namespace fhtdp
