// The main problem of Sec. 2.3 on one image: row smoothing (step 1), the band
// FHTs, the DP with bend-angle windows (step 2) and the read-back (step 3).
// Host side only: the window table and the sequence of launches.
#include <cmath>

#include "common.cuh"

namespace fhtdp {

// Fig. 5: a link of displacement d over n rows has inclination atan(d / n);
// the bend angle between links d and e is |atan(e / n) - atan(d / n)|.  As
// atan is increasing, the admissible e for one d form an interval (the
// union of the ranges of Eqs. 6 and 7), and both of its ends are
// non-decreasing in d, so one sweep with two pointers finds every interval.
// The comparison is the definition itself, evaluated in double.
bool make_angle_table(int n, double gamma, WindowTable *t) {
    if (!(gamma >= 0.0) || !std::isfinite(gamma) || n < 1 || 2 * n - 1 > kMaxD) return false;
    const int D = 2 * n - 1;
    double a[kMaxD];
    for (int i = 0; i < D; ++i) a[i] = std::atan((double)(i - (n - 1)) / n);
    int lo = 0, hi = 0, maxlen = 1;
    for (int i = 0; i < D; ++i) {
        while (a[i] - a[lo] > gamma) ++lo;
        if (hi < i) hi = i;
        while (hi + 1 < D && a[hi + 1] - a[i] <= gamma) ++hi;
        t->lo[i] = (int16_t)(lo - (n - 1));
        t->hi[i] = (int16_t)(hi - (n - 1));
        if (hi - lo + 1 > maxlen) maxlen = hi - lo + 1;
    }
    for (int i = D; i < kMaxD; ++i) t->lo[i] = t->hi[i] = 0;
    t->n = n;
    t->maxlen = maxlen;
    return true;
}

namespace {
constexpr size_t kAngleHead = 256;   // the argmax key, cleared by every call

size_t round_up(size_t v) { return (v + 255) & ~(size_t)255; }

// The smoothed image is stored only for one-row bands (otherwise the
// smoothing is part of the first FHT level).
size_t smooth_bytes(const Shape &s) { return s.n == 1 ? round_up((size_t)s.h * s.w * 4) : 0; }
}  // namespace

// [head][smoothed image h*w, n = 1 only][Hough/V k*2n*W][FHT scratch, same]
// (4-byte values: int32 for integer images, float for float ones)
size_t angle_workspace_bytes(const Shape &s) {
    const size_t hough = (size_t)s.k * 2 * s.n * s.W * 4;
    return kAngleHead + smooth_bytes(s) + 2 * round_up(hough);
}

namespace {
// The launches of detect_angle for one value type: Acc = int32_t for integer
// images (In = uint8_t or int32_t), float for float32 images.
template <typename In, typename Acc>
int detect_angle_t(const In *img, int pitch, const Shape &s, int r, const WindowTable &t,
                   int32_t *x_out, int32_t *d_out, Acc *score_out, void *ws,
                   cudaStream_t stream, const PointMask *pm) {
    char *base = (char *)ws;
    unsigned long long *key = (unsigned long long *)base;
    Acc *smooth = (Acc *)(base + kAngleHead);
    Acc *H = (Acc *)(base + kAngleHead + smooth_bytes(s));
    Acc *tmp = H + round_up((size_t)s.k * 2 * s.n * s.W * 4) / 4;
    int st = cuda_status(cudaMemsetAsync(base, 0, kAngleHead, stream), "cudaMemsetAsync");
    if (st) return st;
    if (r == 0) {   // no smoothing: the FHT reads the image itself
        st = launch_fht_stages<In, Acc>(img, pitch, s, H, tmp, stream);
    } else if (s.n >= 2) {   // smoothing fused into the first FHT level
        st = launch_fht_stages_gauss<In, Acc>(img, pitch, s, r, H, tmp, stream);
    } else {   // one-row bands: smooth into the workspace, then the FHT
        st = launch_gauss_rows<In, Acc>(img, pitch, s.h, s.w, r, smooth, stream);
        if (!st) st = launch_fht_stages<Acc, Acc>(smooth, s.w, s, H, tmp, stream);
    }
    if (!st) st = launch_dp_window<Acc>(H, s, t, stream, pm);
    if (!st) st = launch_backtrack_angle_key<Acc>(H, s, t, key, x_out, d_out, score_out, stream);
    return st;
}
}  // namespace

// pm (optional): Subproblem 3, the polyline must pass the point (the DP
// marks P's band off the point dead).
int detect_angle(const void *img, int dtype, int pitch, const Shape &s, int r,
                 const WindowTable &t, int32_t *x_out, int32_t *d_out, void *score_out,
                 void *ws, cudaStream_t stream, const PointMask *pm) {
    if (dtype == FHTDP_U8)
        return detect_angle_t<uint8_t, int32_t>((const uint8_t *)img, pitch, s, r, t, x_out,
                                                d_out, (int32_t *)score_out, ws, stream, pm);
    if (dtype == FHTDP_I32)
        return detect_angle_t<int32_t, int32_t>((const int32_t *)img, pitch, s, r, t, x_out,
                                                d_out, (int32_t *)score_out, ws, stream, pm);
    return detect_angle_t<float, float>((const float *)img, pitch, s, r, t, x_out, d_out,
                                        (float *)score_out, ws, stream, pm);
}

}  // namespace fhtdp
