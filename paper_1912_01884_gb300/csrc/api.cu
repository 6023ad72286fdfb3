// C-ABI entry points: argument validation, dispatch on the pixel type, and
// error reporting.  No exception and no allocation happens here.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>

#include "common.cuh"
#include "cnn.cuh"
#include "engine.cuh"

namespace fhtdp {

namespace {
thread_local char g_last_error[512] = "";
std::atomic<uint64_t> g_launches{0};
}  // namespace

int launched(const char *what) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cuda_status(cudaGetLastError(), what);
}

void clear_error() { g_last_error[0] = 0; }

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_status(cudaError_t err, const char *what) {
    if (err == cudaSuccess) return FHTDP_OK;
    return set_error(FHTDP_ECUDA, "%s: %s", what, cudaGetErrorString(err));
}

bool make_shape(int h, int w, int k, Shape *out) {
    if (h < 1 || w < 1 || k < 1 || h % k != 0) return false;
    int n = h / k;
    if (n > 256 || (n & (n - 1)) != 0) return false;
    if (w > (1 << 20) || h > (1 << 20)) return false;
    Shape s;
    s.h = h;
    s.w = w;
    s.k = k;
    s.n = n;
    s.W = w + n;
    s.D = 2 * n - 1;
    s.log2n = 0;
    while ((1 << s.log2n) < n) ++s.log2n;
    s.vw = w;
    *out = s;
    return true;
}

namespace {

int bad_shape(int h, int w, int k) {
    return set_error(FHTDP_EINVAL,
                     "invalid shape h=%d w=%d k=%d: need h = k*n with n a power of two "
                     "in [1, 256], 1 <= w <= 2^20, h <= 2^20",
                     h, w, k);
}

bool valid_dtype(int dtype) { return dtype == FHTDP_U8 || dtype == FHTDP_I32 || dtype == FHTDP_F32; }

size_t hough_elems(const Shape &s) { return (size_t)s.k * 2 * s.n * s.W; }

}  // namespace
}  // namespace fhtdp

using namespace fhtdp;

extern "C" {

const char *fhtdp_last_error(void) { return g_last_error; }

int fhtdp_version(void) { return 100; }

uint64_t fhtdp_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

size_t fhtdp_hough_bytes(int dtype, int h, int w, int k) {
    Shape s;
    if (!valid_dtype(dtype) || !make_shape(h, w, k, &s)) return 0;
    return hough_elems(s) * 4;
}

size_t fhtdp_fht_workspace_bytes(int dtype, int h, int w, int k) {
    Shape s;
    if (!valid_dtype(dtype) || !make_shape(h, w, k, &s)) return 0;
    return s.log2n >= 2 ? hough_elems(s) * 4 : 0;
}

int fhtdp_fht_bands(const void *img, int dtype, int h, int w, int pitch, int k, void *hough,
                    void *ws, size_t ws_bytes, cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (!make_shape(h, w, k, &s)) return bad_shape(h, w, k);
    if (pitch < w) return set_error(FHTDP_EINVAL, "pitch %d < w %d", pitch, w);
    if (!img || !hough) return set_error(FHTDP_EINVAL, "null img or hough pointer");
    size_t need = fhtdp_fht_workspace_bytes(dtype, h, w, k);
    if (need && (!ws || ws_bytes < need))
        return set_error(FHTDP_EWORKSPACE, "fht workspace needs %zu bytes, got %zu", need,
                         ws ? ws_bytes : (size_t)0);
    switch (dtype) {
        case FHTDP_U8:
            return launch_fht_stages<uint8_t, int32_t>((const uint8_t *)img, pitch, s,
                                                       (int32_t *)hough, (int32_t *)ws, stream);
        case FHTDP_I32:
            return launch_fht_stages<int32_t, int32_t>((const int32_t *)img, pitch, s,
                                                       (int32_t *)hough, (int32_t *)ws, stream);
        default:
            return launch_fht_stages<float, float>((const float *)img, pitch, s, (float *)hough,
                                                   (float *)ws, stream);
    }
}

int fhtdp_polyline_dp(void *hough, int dtype, int h, int w, int k, int B, cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (!make_shape(h, w, k, &s)) return bad_shape(h, w, k);
    if (B < 0) return set_error(FHTDP_EINVAL, "bend limit B=%d < 0", B);
    if (!hough) return set_error(FHTDP_EINVAL, "null hough pointer");
    if (dtype == FHTDP_F32) return launch_dp_inplace<float>((float *)hough, s, B, stream);
    return launch_dp_inplace<int32_t>((int32_t *)hough, s, B, stream);
}

int fhtdp_backtrack(const void *V, int dtype, int h, int w, int k, int B, int32_t *x_out,
                    int32_t *d_out, void *score_out, cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (!make_shape(h, w, k, &s)) return bad_shape(h, w, k);
    if (B < 0) return set_error(FHTDP_EINVAL, "bend limit B=%d < 0", B);
    if (!V || !x_out || !d_out || !score_out)
        return set_error(FHTDP_EINVAL, "null V or output pointer");
    if (dtype == FHTDP_F32)
        return launch_backtrack<float>((const float *)V, s, B, x_out, d_out, (float *)score_out,
                                       stream);
    return launch_backtrack<int32_t>((const int32_t *)V, s, B, x_out, d_out,
                                     (int32_t *)score_out, stream);
}

size_t fhtdp_workspace_bytes(int dtype, int h, int w, int k, int B) {
    Shape s;
    if (!valid_dtype(dtype) || !make_shape(h, w, k, &s) || B < 0) return 0;
    return engine_workspace_bytes(dtype, s, B);
}

int fhtdp_detect_polyline(const void *img, int dtype, int h, int w, int pitch, int k, int B,
                          int32_t *x_out, int32_t *d_out, void *score_out, void *ws,
                          size_t ws_bytes, cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (!make_shape(h, w, k, &s)) return bad_shape(h, w, k);
    if (pitch < w) return set_error(FHTDP_EINVAL, "pitch %d < w %d", pitch, w);
    if (B < 0) return set_error(FHTDP_EINVAL, "bend limit B=%d < 0", B);
    if (!img || !x_out || !d_out || !score_out)
        return set_error(FHTDP_EINVAL, "null image or output pointer");
    size_t need = engine_workspace_bytes(dtype, s, B);
    if (!ws || ws_bytes < need)
        return set_error(FHTDP_EWORKSPACE, "workspace needs %zu bytes, got %zu", need,
                         ws ? ws_bytes : (size_t)0);
    return engine_detect(img, dtype, pitch, s, B, x_out, d_out, score_out, ws, ws_bytes, stream);
}

// ---------------------------------------------------------------------------
// The main problem (Sec. 2.3): smoothing and bend-angle windows.
namespace {
int check_angle_common(int dtype, int h, int w, int k, double gamma, Shape *s) {
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (!make_shape(h, w, k, s)) return bad_shape(h, w, k);
    if (!(gamma >= 0.0) || !std::isfinite(gamma))
        return set_error(FHTDP_EINVAL, "bend angle gamma must be finite and >= 0");
    return FHTDP_OK;
}
int check_gauss(int dtype, int h, int r) {
    if (r < 0 || r > kMaxGaussR)
        return set_error(FHTDP_EINVAL, "smoothing half-width r=%d outside [0, %d]", r, kMaxGaussR);
    if (dtype == FHTDP_U8 && 255.0 * std::ldexp(1.0, 2 * r) * h >= 2147483648.0)
        return set_error(FHTDP_EINVAL, "255 * 4^r * h >= 2^31: int32 sums could overflow");
    return FHTDP_OK;
}
}  // namespace

int fhtdp_angle_window(int n, double gamma, int32_t *lohi) {
    g_last_error[0] = 0;
    if (n < 1 || n > 256 || (n & (n - 1)) || !lohi)
        return set_error(FHTDP_EINVAL, "angle window: n a power of two in [1, 256], non-null lohi");
    WindowTable t;
    if (!make_angle_table(n, gamma, &t))
        return set_error(FHTDP_EINVAL, "bend angle gamma must be finite and >= 0");
    for (int i = 0; i < 2 * n - 1; ++i) {
        lohi[2 * i] = t.lo[i];
        lohi[2 * i + 1] = t.hi[i];
    }
    return FHTDP_OK;
}

int fhtdp_gauss_rows(const void *img, int dtype, int h, int w, int pitch, int r, void *out,
                     cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (h < 1 || w < 1 || h > (1 << 20) || w > (1 << 20))
        return set_error(FHTDP_EINVAL, "invalid image %d x %d", h, w);
    if (pitch < w) return set_error(FHTDP_EINVAL, "pitch %d < w %d", pitch, w);
    if (!img || !out) return set_error(FHTDP_EINVAL, "null img or out pointer");
    int st = check_gauss(dtype, h, r);
    if (st) return st;
    if (dtype == FHTDP_U8)
        return launch_gauss_rows<uint8_t, int32_t>((const uint8_t *)img, pitch, h, w, r,
                                                   (int32_t *)out, stream);
    if (dtype == FHTDP_I32)
        return launch_gauss_rows<int32_t, int32_t>((const int32_t *)img, pitch, h, w, r,
                                                   (int32_t *)out, stream);
    return launch_gauss_rows<float, float>((const float *)img, pitch, h, w, r, (float *)out,
                                           stream);
}

int fhtdp_polyline_dp_angle(void *hough, int dtype, int h, int w, int k, double gamma,
                            cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    int st = check_angle_common(dtype, h, w, k, gamma, &s);
    if (st) return st;
    if (!hough) return set_error(FHTDP_EINVAL, "null hough pointer");
    WindowTable t;
    make_angle_table(s.n, gamma, &t);
    if (dtype == FHTDP_F32) return launch_dp_window<float>((float *)hough, s, t, stream);
    return launch_dp_window<int32_t>((int32_t *)hough, s, t, stream);
}

int fhtdp_backtrack_angle(const void *V, int dtype, int h, int w, int k, double gamma,
                          int32_t *x_out, int32_t *d_out, void *score_out, cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    int st = check_angle_common(dtype, h, w, k, gamma, &s);
    if (st) return st;
    if (!V || !x_out || !d_out || !score_out)
        return set_error(FHTDP_EINVAL, "null V or output pointer");
    WindowTable t;
    make_angle_table(s.n, gamma, &t);
    if (dtype == FHTDP_F32)
        return launch_backtrack_angle<float>((const float *)V, s, t, x_out, d_out,
                                             (float *)score_out, stream);
    return launch_backtrack_angle<int32_t>((const int32_t *)V, s, t, x_out, d_out,
                                           (int32_t *)score_out, stream);
}

size_t fhtdp_angle_workspace_bytes(int dtype, int h, int w, int k, int r) {
    Shape s;
    if (!valid_dtype(dtype) || !make_shape(h, w, k, &s) || r < 0 || r > kMaxGaussR) return 0;
    return angle_workspace_bytes(s);
}

int fhtdp_detect_polyline_angle(const void *img, int dtype, int h, int w, int pitch, int k,
                                int r, double gamma, int32_t *x_out, int32_t *d_out,
                                void *score_out, void *ws, size_t ws_bytes, cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    int st = check_angle_common(dtype, h, w, k, gamma, &s);
    if (st) return st;
    if (pitch < w) return set_error(FHTDP_EINVAL, "pitch %d < w %d", pitch, w);
    st = check_gauss(dtype, h, r);
    if (st) return st;
    if (!img || !x_out || !d_out || !score_out)
        return set_error(FHTDP_EINVAL, "null image or output pointer");
    size_t need = angle_workspace_bytes(s);
    if (!ws || ws_bytes < need)
        return set_error(FHTDP_EWORKSPACE, "workspace needs %zu bytes, got %zu", need,
                         ws ? ws_bytes : (size_t)0);
    WindowTable t;
    make_angle_table(s.n, gamma, &t);
    return detect_angle(img, dtype, pitch, s, r, t, x_out, d_out, score_out, ws, stream);
}

int fhtdp_detect_through_point_angle(const void *img, int dtype, int h, int w, int pitch, int k,
                                     int r, double gamma, int j, int xp, int32_t *x_out,
                                     int32_t *d_out, void *score_out, void *ws, size_t ws_bytes,
                                     cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    int st = check_angle_common(dtype, h, w, k, gamma, &s);
    if (st) return st;
    if (pitch < w) return set_error(FHTDP_EINVAL, "pitch %d < w %d", pitch, w);
    st = check_gauss(dtype, h, r);
    if (st) return st;
    if (j < 0 || j > k || xp < 0 || xp >= w)
        return set_error(FHTDP_EINVAL, "point (%d, border %d) outside [0, %d) x [0, %d]", xp, j,
                         w, k);
    if (!img || !x_out || !d_out || !score_out)
        return set_error(FHTDP_EINVAL, "null image or output pointer");
    size_t need = angle_workspace_bytes(s);
    if (!ws || ws_bytes < need)
        return set_error(FHTDP_EWORKSPACE, "workspace needs %zu bytes, got %zu", need,
                         ws ? ws_bytes : (size_t)0);
    WindowTable t;
    make_angle_table(s.n, gamma, &t);
    const PointMask pm{j, xp};
    return detect_angle(img, dtype, pitch, s, r, t, x_out, d_out, score_out, ws, stream, &pm);
}

// ---------------------------------------------------------------------------
// Subproblems 2-3: the extreme polyline through a given point.
size_t fhtdp_through_workspace_bytes(int dtype, int h, int w, int k) {
    Shape s;
    if (!valid_dtype(dtype) || !make_shape(h, w, k, &s)) return 0;
    return through_workspace_bytes(s);
}

int fhtdp_detect_through_point(const void *img, int dtype, int h, int w, int pitch, int k, int B,
                               int j, int xp, int32_t *x_out, int32_t *d_out, void *score_out,
                               void *ws, size_t ws_bytes, cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (!make_shape(h, w, k, &s)) return bad_shape(h, w, k);
    if (pitch < w) return set_error(FHTDP_EINVAL, "pitch %d < w %d", pitch, w);
    if (B < 0) return set_error(FHTDP_EINVAL, "bend limit B=%d < 0", B);
    if (j < 0 || j > k || xp < 0 || xp >= w)
        return set_error(FHTDP_EINVAL, "point (%d, border %d) outside [0, %d) x [0, %d]", xp, j,
                         w, k);
    if (!img || !x_out || !d_out || !score_out)
        return set_error(FHTDP_EINVAL, "null image or output pointer");
    size_t need = through_workspace_bytes(s);
    if (!ws || ws_bytes < need)
        return set_error(FHTDP_EWORKSPACE, "workspace needs %zu bytes, got %zu", need,
                         ws ? ws_bytes : (size_t)0);
    const PointMask pm{j, xp};
    return detect_through(img, dtype, pitch, s, B, pm, x_out, d_out, score_out, ws, stream);
}

// ---------------------------------------------------------------------------
// Vertices in the zero padding (Sec. 2.2).
int fhtdp_detect_polyline_padded(const void *img, int dtype, int h, int w, int pitch, int k,
                                 int B, int32_t *x_out, int32_t *d_out, void *score_out,
                                 void *ws, size_t ws_bytes, cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (!make_shape(h, w, k, &s)) return bad_shape(h, w, k);
    if (pitch < w) return set_error(FHTDP_EINVAL, "pitch %d < w %d", pitch, w);
    if (B < 0) return set_error(FHTDP_EINVAL, "bend limit B=%d < 0", B);
    if (!img || !x_out || !d_out || !score_out)
        return set_error(FHTDP_EINVAL, "null image or output pointer");
    size_t need = through_workspace_bytes(s);
    if (!ws || ws_bytes < need)
        return set_error(FHTDP_EWORKSPACE, "workspace needs %zu bytes, got %zu", need,
                         ws ? ws_bytes : (size_t)0);
    s.vw = s.W;
    return detect_padded(img, dtype, pitch, s, B, x_out, d_out, score_out, ws, stream);
}

// ---------------------------------------------------------------------------
// Two different extreme polylines (Sec. 3, Figs. 6d and 7a).
size_t fhtdp_two_workspace_bytes(int dtype, int h, int w, int k) {
    return fhtdp_through_workspace_bytes(dtype, h, w, k);
}

int fhtdp_detect_two_polylines(const void *img, int dtype, int h, int w, int pitch, int k, int B,
                               int sep, int32_t *x_out, int32_t *d_out, void *score_out,
                               void *ws, size_t ws_bytes, cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (!make_shape(h, w, k, &s)) return bad_shape(h, w, k);
    if (pitch < w) return set_error(FHTDP_EINVAL, "pitch %d < w %d", pitch, w);
    if (B < 0) return set_error(FHTDP_EINVAL, "bend limit B=%d < 0", B);
    if (sep < 1) return set_error(FHTDP_EINVAL, "separation %d < 1", sep);
    if (!img || !x_out || !d_out || !score_out)
        return set_error(FHTDP_EINVAL, "null image or output pointer");
    size_t need = through_workspace_bytes(s);
    if (!ws || ws_bytes < need)
        return set_error(FHTDP_EWORKSPACE, "workspace needs %zu bytes, got %zu", need,
                         ws ? ws_bytes : (size_t)0);
    return detect_two(img, dtype, pitch, s, B, sep, x_out, d_out, score_out, ws, stream);
}

// ---------------------------------------------------------------------------
// Mostly horizontal curves (Sec. 3, Fig. 7): the image transposed into the
// workspace, then the fused engine.
namespace {
int transposed_pitch(int h) { return (h + 63) / 64 * 64; }
size_t transposed_bytes(int dtype, int h, int w) {
    const size_t b = (size_t)w * transposed_pitch(h) * (dtype == FHTDP_U8 ? 1 : 4);
    return (b + 255) & ~(size_t)255;
}
}  // namespace

int fhtdp_transpose(const void *src, int dtype, int h, int w, int pitch, void *dst, int dpitch,
                    cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (h < 1 || w < 1 || h > (1 << 20) || w > (1 << 20))
        return set_error(FHTDP_EINVAL, "invalid image %d x %d", h, w);
    if (pitch < w || dpitch < h)
        return set_error(FHTDP_EINVAL, "pitch %d < w %d or dst pitch %d < h %d", pitch, w,
                         dpitch, h);
    if (!src || !dst || src == dst) return set_error(FHTDP_EINVAL, "null or aliased buffers");
    switch (dtype) {
        case FHTDP_U8:
            return launch_transpose<uint8_t>((const uint8_t *)src, h, w, pitch, (uint8_t *)dst,
                                             dpitch, stream);
        case FHTDP_I32:
            return launch_transpose<int32_t>((const int32_t *)src, h, w, pitch, (int32_t *)dst,
                                             dpitch, stream);
        default:
            return launch_transpose<float>((const float *)src, h, w, pitch, (float *)dst, dpitch,
                                           stream);
    }
}

size_t fhtdp_horizontal_workspace_bytes(int dtype, int h, int w, int k, int B) {
    Shape s;
    if (!valid_dtype(dtype) || !make_shape(w, h, k, &s) || B < 0) return 0;
    return transposed_bytes(dtype, h, w) + engine_workspace_bytes(dtype, s, B);
}

int fhtdp_detect_polyline_horizontal(const void *img, int dtype, int h, int w, int pitch, int k,
                                     int B, int32_t *y_out, int32_t *d_out, void *score_out,
                                     void *ws, size_t ws_bytes, cudaStream_t stream) {
    g_last_error[0] = 0;
    Shape s;
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (!make_shape(w, h, k, &s))
        return set_error(FHTDP_EINVAL,
                         "invalid shape h=%d w=%d k=%d: horizontal bands need w = k*n with n a "
                         "power of two in [1, 256], 1 <= h <= 2^20, w <= 2^20",
                         h, w, k);
    if (pitch < w) return set_error(FHTDP_EINVAL, "pitch %d < w %d", pitch, w);
    if (B < 0) return set_error(FHTDP_EINVAL, "bend limit B=%d < 0", B);
    if (!img || !y_out || !d_out || !score_out)
        return set_error(FHTDP_EINVAL, "null image or output pointer");
    const size_t tb = transposed_bytes(dtype, h, w);
    const size_t need = tb + engine_workspace_bytes(dtype, s, B);
    if (!ws || ws_bytes < need)
        return set_error(FHTDP_EWORKSPACE, "workspace needs %zu bytes, got %zu", need,
                         ws ? ws_bytes : (size_t)0);
    const int tp = transposed_pitch(h);
    int st;
    switch (dtype) {
        case FHTDP_U8:
            st = launch_transpose<uint8_t>((const uint8_t *)img, h, w, pitch, (uint8_t *)ws, tp,
                                           stream);
            break;
        case FHTDP_I32:
            st = launch_transpose<int32_t>((const int32_t *)img, h, w, pitch, (int32_t *)ws, tp,
                                           stream);
            break;
        default:
            st = launch_transpose<float>((const float *)img, h, w, pitch, (float *)ws, tp, stream);
    }
    if (st) return st;
    return engine_detect(ws, dtype, tp, s, B, y_out, d_out, score_out, (char *)ws + tb,
                         ws_bytes - tb, stream);
}

// ---------------------------------------------------------------------------
// Learned window proposal.
int fhtdp_cnn_downsample4(const uint8_t *img, int n, int h, int w, void *out,
                          cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!img || !out || n < 1 || h < 4 || w < 4 || h % 4 || w % 4)
        return set_error(FHTDP_EINVAL, "downsample: need h, w multiples of 4 and non-null buffers");
    return cnn_downsample4(img, n, h, w, out, stream);
}

int fhtdp_cnn_conv3x3(const void *x, int cin, int n, int h, int w, int dil, const void *wt,
                      const float *bias, int relu, void *y, cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!x || !wt || !y || n < 1 || (cin != 1 && cin != 32) || !cnn_shape_ok(h, w, dil))
        return set_error(FHTDP_EINVAL,
                         "conv3x3: need cin 1 or 32, w a multiple of 64, 1 <= dil <= 8");
    return cnn_conv3x3(x, cin, n, h, w, dil, wt, bias, relu, y, stream);
}

int fhtdp_cnn_status(int clear) {
    g_last_error[0] = 0;
    const int st = cnn_tc_status(clear);
    return st == FHTDP_ECUDA ? -FHTDP_ECUDA : st;
}

int fhtdp_cnn_conv3x3_dgrad(const void *dz, int n, int h, int w, int dil, const void *wt,
                            void *wflip, void *dx, cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!dz || !wt || !wflip || !dx || n < 1 || !cnn_shape_ok(h, w, dil))
        return set_error(FHTDP_EINVAL, "conv3x3_dgrad: bad arguments");
    int st = cnn_flip_transpose(wt, wflip, stream);
    if (st) return st;
    return cnn_conv3x3(dz, 32, n, h, w, dil, wflip, nullptr, 0, dx, stream);
}

int fhtdp_cnn_relu_backward(const void *y, void *dy, long long count, cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!y || !dy || count < 0) return set_error(FHTDP_EINVAL, "relu_backward: bad arguments");
    return cnn_relu_backward(y, dy, count, stream);
}

int fhtdp_cnn_conv3x3_wgrad(const void *x, int cin, int n, int h, int w, int dil, const void *dz,
                            float *dw, float *db, cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!x || !dz || !dw || n < 1 || (cin != 1 && cin != 32) || !cnn_shape_ok(h, w, dil))
        return set_error(FHTDP_EINVAL, "conv3x3_wgrad: bad arguments");
    return cnn_wgrad(x, cin, n, h, w, dil, dz, dw, db, stream);
}

int fhtdp_cnn_band_head(const void *logits, int n, int h, int w, int bands,
                        const int32_t *labels, float scale, void *dlogits, float *loss,
                        int32_t *pred, cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!logits || n < 1 || bands < 1 || h % bands || w < 1)
        return set_error(FHTDP_EINVAL, "band_head: bad arguments");
    return cnn_band_head(logits, n, h, w, bands, labels, scale, dlogits, loss, pred, stream);
}

int fhtdp_cnn_adam(float *p, float *m, float *v, const float *g, int count, float lr, float b1,
                   float b2, float eps, int step, void *wb, cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!p || !m || !v || !g || count < 1 || step < 1)
        return set_error(FHTDP_EINVAL, "adam: bad arguments");
    return cnn_adam(p, m, v, g, count, lr, b1, b2, eps, step, wb, stream);
}

int fhtdp_cnn_to_bf16(const float *src, void *dst, int count, cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!src || !dst || count < 1) return set_error(FHTDP_EINVAL, "to_bf16: bad arguments");
    return cnn_to_bf16(src, dst, count, stream);
}

int fhtdp_cnn_bin_windows(const int32_t *pred, int count, int n, int margin, int32_t *win,
                          cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!pred || !win || count < 1 || n < 1 || margin < 0)
        return set_error(FHTDP_EINVAL, "bin_windows: bad arguments");
    return cnn_bin_windows(pred, count, n, margin, win, stream);
}

void fhtdp_debug_inject(int band, int tile, long long wait_cycles) {
    debug_inject(band, tile, wait_cycles);
}

int fhtdp_workspace_status(const void *ws, cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!ws) return set_error(FHTDP_EINVAL, "null workspace");
    return engine_status(ws, stream);
}

struct fhtdp_batch_plan {
    BatchPlan *impl;
};

int fhtdp_batch_plan_create(const fhtdp_image *images, int count, int dtype,
                            fhtdp_batch_plan **plan_out) {
    g_last_error[0] = 0;
    if (!plan_out) return set_error(FHTDP_EINVAL, "null plan_out");
    *plan_out = nullptr;
    if (!valid_dtype(dtype)) return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    BatchPlan *impl = nullptr;
    int st = batch_create(images, count, dtype, &impl);
    if (st) return st;
    fhtdp_batch_plan *p = new (std::nothrow) fhtdp_batch_plan{impl};
    if (!p) {
        batch_destroy(impl);
        return set_error(FHTDP_EINVAL, "out of host memory");
    }
    *plan_out = p;
    return FHTDP_OK;
}

size_t fhtdp_batch_workspace_bytes(const fhtdp_batch_plan *plan) {
    return plan ? batch_workspace_bytes(plan->impl) : 0;
}

long long fhtdp_batch_items(const fhtdp_batch_plan *plan) {
    return plan ? batch_items(plan->impl) : 0;
}

int fhtdp_batch_upload(fhtdp_batch_plan *plan, void *ws, size_t ws_bytes, cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!plan) return set_error(FHTDP_EINVAL, "null plan");
    return batch_upload(plan->impl, ws, ws_bytes, stream);
}

int fhtdp_batch_run(const fhtdp_batch_plan *plan, void *ws, cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!plan) return set_error(FHTDP_EINVAL, "null plan");
    return batch_run(plan->impl, ws, stream);
}

int fhtdp_batch_autotune(fhtdp_batch_plan *plan, void *ws, int reps, cudaStream_t stream,
                         long long *target_out) {
    g_last_error[0] = 0;
    if (!plan) return set_error(FHTDP_EINVAL, "null plan");
    return batch_autotune(plan->impl, ws, reps, stream, target_out);
}

int fhtdp_batch_choice(const fhtdp_batch_plan *plan, int n, int *mode, long long *target,
                       int *tile, int *depth) {
    g_last_error[0] = 0;
    if (!plan) return set_error(FHTDP_EINVAL, "null plan");
    batch_choice(plan->impl, n, mode, target, tile, depth);
    return FHTDP_OK;
}

int fhtdp_batch_configure(fhtdp_batch_plan *plan, void *ws, int n, int tile, int depth,
                          cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!plan) return set_error(FHTDP_EINVAL, "null plan");
    return batch_configure(plan->impl, ws, n, tile, depth, stream);
}

int fhtdp_batch_points(fhtdp_batch_plan *plan, void *ws, const int32_t *points,
                       cudaStream_t stream) {
    g_last_error[0] = 0;
    if (!plan) return set_error(FHTDP_EINVAL, "null plan");
    return batch_points(plan->impl, ws, points, stream);
}

int fhtdp_batch_angle(fhtdp_batch_plan *plan, double gamma) {
    g_last_error[0] = 0;
    if (!plan) return set_error(FHTDP_EINVAL, "null plan");
    return batch_angle(plan->impl, gamma);
}

void fhtdp_batch_plan_destroy(fhtdp_batch_plan *plan) {
    if (!plan) return;
    batch_destroy(plan->impl);
    delete plan;
}

}  // extern "C"
