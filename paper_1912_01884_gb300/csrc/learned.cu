// The learned window proposal as library calls: the CNN's parameter block,
// its initialisation, forward and backward passes and Adam step, and the
// proposal-then-pruned-DP detection with the full DP as a device-side
// fallback.  The paper has no counterpart: this is an addition in front of
// the exact method, whose results it keeps wherever it is not sure.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "cnn.cuh"
#include "engine.cuh"

namespace fhtdp {
namespace {

constexpr int kC = 32;
constexpr int kLayers = 4;
constexpr int kDil[kLayers] = {1, 2, 4, 8};

// Rows of a layer's weight matrix: taps x input channels (layer 0: 16 rows,
// taps 9..15 zero).
constexpr int taps_rows(int l) { return l == 0 ? 16 : 9 * kC; }

// Parameter block: per layer, FP32 weights [rows][32], FP32 bias [32], Adam
// moments of both, and the bf16 weight copy the forward pass reads.
struct LayerOff {
    size_t w, b, mw, vw, mb, vb, w16;
};
size_t align256(size_t v) { return (v + 255) / 256 * 256; }
LayerOff layer_off(int l, size_t *end = nullptr) {
    size_t o = 0;
    LayerOff r{};
    for (int i = 0; i <= l; ++i) {
        const size_t nw = (size_t)taps_rows(i) * kC;
        r.w = o;
        o = align256(o + nw * 4);
        r.b = o;
        o = align256(o + kC * 4);
        r.mw = o;
        o = align256(o + nw * 4);
        r.vw = o;
        o = align256(o + nw * 4);
        r.mb = o;
        o = align256(o + kC * 4);
        r.vb = o;
        o = align256(o + kC * 4);
        r.w16 = o;
        o = align256(o + nw * 2);
    }
    if (end) *end = o;
    return r;
}
size_t param_bytes() {
    size_t end = 0;
    layer_off(kLayers - 1, &end);
    return end;
}

// CNN workspace for n images of h x w pixels (low-resolution ho x wo): the
// input, the four layer outputs, two gradient buffers, the flipped weights,
// the FP32 gradients of every layer and the loss.
struct CnnWs {
    size_t x0, act[kLayers], g0, g1, wflip, grads[kLayers], loss, total;
};
CnnWs cnn_ws(int n, int h, int w) {
    const size_t px = (size_t)n * (h / 4) * (w / 4);
    CnnWs c{};
    size_t o = 0;
    c.x0 = o;
    o = align256(o + px * 2);
    for (int l = 0; l < kLayers; ++l) {
        c.act[l] = o;
        o = align256(o + px * kC * 2);
    }
    c.g0 = o;
    o = align256(o + px * kC * 2);
    c.g1 = o;
    o = align256(o + px * kC * 2);
    c.wflip = o;
    o = align256(o + 9 * kC * kC * 2);
    for (int l = 0; l < kLayers; ++l) {
        c.grads[l] = o;
        o = align256(o + ((size_t)taps_rows(l) * kC + kC) * 4);
    }
    c.loss = o;
    o = align256(o + 4);
    c.total = o;
    return c;
}

// Inference only: the input and two alternating activation buffers.
CnnWs cnn_ws_infer(int n, int h, int w) {
    const size_t px = (size_t)n * (h / 4) * (w / 4);
    CnnWs c{};
    size_t o = 0;
    c.x0 = o;
    o = align256(o + px * 2);
    for (int l = 0; l < 2; ++l) {
        c.act[l] = o;
        o = align256(o + px * kC * 2);
    }
    c.total = o;
    return c;
}

bool cnn_dims_ok(int n, int h, int w, int bands) {
    return n >= 1 && bands >= 1 && h % 4 == 0 && w % 4 == 0 && (h / 4) % bands == 0 &&
           cnn_shape_ok(h / 4, w / 4, 8);
}

int forward(const char *P, const uint8_t *imgs, int n, int h, int w, int bands, char *ws,
            const CnnWs &c, int32_t *pred, float *conf, bool keep, cudaStream_t stream) {
    const int ho = h / 4, wo = w / 4;
    int st = cnn_downsample4(imgs, n, h, w, ws + c.x0, stream);
    const void *in = ws + c.x0;
    for (int l = 0; l < kLayers && !st; ++l) {
        const LayerOff o = layer_off(l);
        // without `keep` (inference) two buffers alternate
        void *out = ws + c.act[keep ? l : (l & 1)];
        st = cnn_conv3x3(in, l == 0 ? 1 : kC, n, ho, wo, kDil[l], P + o.w16,
                         (const float *)(P + o.b), l + 1 < kLayers ? 1 : 0, out, stream);
        in = out;
    }
    if (!st)
        st = cnn_band_head(in, n, ho, wo, bands, nullptr, 0.0f, nullptr, nullptr, pred, stream,
                           conf);
    return st;
}

// ---------------------------------------------------------------------------
// The fallback decision of the learned detection: image i falls back to the
// full DP when its pruned DP found no polyline inside the windows, when the
// polyline touches a window edge that is not an edge of the displacement
// range (a better link may lie just outside), when its score is below
// margin * h (the confidence margin, in mean intensity per image row), or
// when the network gave some band's bin a softmax probability below
// min_conf.
__global__ void decide_kernel(int N, int k, int n, int h, float margin, float min_conf,
                              const int32_t *__restrict__ x, const int32_t *__restrict__ d,
                              const int32_t *__restrict__ s, const int32_t *__restrict__ win,
                              const float *__restrict__ conf, int32_t *__restrict__ fb,
                              int32_t *__restrict__ used) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        bool f = x[(size_t)i * (k + 1)] < 0 || (float)s[i] < margin * (float)h;
        for (int b = 0; b < k && !f; ++b) f = conf[(size_t)i * k + b] < min_conf;
        for (int b = 0; b < k && !f; ++b) {
            const int lo = win[((size_t)i * k + b) * 2], hi = win[((size_t)i * k + b) * 2 + 1];
            const int db = d[(size_t)i * k + b];
            f = (db == lo && lo > -(n - 1)) || (db == hi && hi < n - 1);
        }
        fb[i] = f ? 1 : 0;
        if (used) used[i] = f ? 1 : 0;
    }
}

// The pruned results of the images that did not fall back, into the
// caller's outputs (out[i] = {x_out, d_out, score_out} of image i).
struct OutPtrs {
    int32_t *x, *d, *s;
};
__global__ void merge_kernel(int N, int k, const int32_t *__restrict__ fb,
                             const int32_t *__restrict__ x, const int32_t *__restrict__ d,
                             const int32_t *__restrict__ s, const OutPtrs *__restrict__ out) {
    const int i = blockIdx.x;
    if (i >= N || fb[i]) return;
    const OutPtrs o = out[i];
    for (int j = threadIdx.x; j <= k; j += blockDim.x) o.x[j] = x[(size_t)i * (k + 1) + j];
    for (int j = threadIdx.x; j < k; j += blockDim.x) o.d[j] = d[(size_t)i * k + j];
    if (threadIdx.x == 0) o.s[0] = s[i];
}

}  // namespace
}  // namespace fhtdp

using namespace fhtdp;

// The learned detection plan: images of one shape, the CNN's chunked
// inference workspace, the pruned-DP batch and the full-DP batch.
struct fhtdp_learned_plan {
    int N, h, w, k, B, half, chunk;
    std::vector<fhtdp_image> io;      // the caller's images and outputs
    BatchPlan *full = nullptr;        // outputs: the caller's; enabled per image
    BatchPlan *pruned = nullptr;      // outputs: scratch; windows from the proposal
    size_t full_bytes = 0;
    // workspace offsets
    size_t off_full, off_pruned, off_cnn, off_pred, off_conf, off_win, off_x, off_d, off_s, off_fb,
        off_out, total;
    CnnWs cws;
    void *bound = nullptr;
    ~fhtdp_learned_plan() {
        if (full) batch_destroy(full);
        if (pruned) batch_destroy(pruned);
    }
};

extern "C" {

size_t fhtdp_cnn_param_bytes(void) { return param_bytes(); }

int fhtdp_cnn_init(void *params, unsigned long long seed, cudaStream_t stream) {
    clear_error();
    if (!params) return set_error(FHTDP_EINVAL, "null params");
    char *P = (char *)params;
    int st = cuda_status(cudaMemsetAsync(P, 0, param_bytes(), stream), "cudaMemsetAsync");
    for (int l = 0; l < kLayers && !st; ++l) {
        const LayerOff o = layer_off(l);
        const int cin = l == 0 ? 1 : kC;
        st = cnn_he_init((float *)(P + o.w), taps_rows(l), kC, l == 0 ? 9 : taps_rows(l),
                         sqrtf(2.0f / (9.0f * cin)), seed * 4 + (unsigned long long)l, stream);
        if (!st)
            st = cnn_to_bf16((const float *)(P + o.w), P + o.w16, taps_rows(l) * kC, stream);
    }
    return st;
}

size_t fhtdp_cnn_workspace_bytes(int n, int h, int w) {
    if (n < 1 || h < 4 || w < 4) return 0;
    return cnn_ws(n, h, w).total;
}

int fhtdp_cnn_forward(const void *params, const uint8_t *imgs, int n, int h, int w, int bands,
                      void *ws, size_t ws_bytes, int32_t *pred, float *conf,
                      cudaStream_t stream) {
    clear_error();
    if (!params || !imgs || !ws || !pred) return set_error(FHTDP_EINVAL, "null pointer");
    if (!cnn_dims_ok(n, h, w, bands))
        return set_error(FHTDP_EINVAL, "unsupported CNN shape n=%d h=%d w=%d bands=%d", n, h, w,
                         bands);
    const CnnWs c = cnn_ws(n, h, w);
    if (ws_bytes < c.total)
        return set_error(FHTDP_EWORKSPACE, "CNN workspace needs %zu bytes, got %zu", c.total,
                         ws_bytes);
    return forward((const char *)params, imgs, n, h, w, bands, (char *)ws, c, pred, conf, true,
                   stream);
}

int fhtdp_cnn_backward(const void *params, const int32_t *labels, int n, int h, int w, int bands,
                       void *ws, size_t ws_bytes, float *loss, cudaStream_t stream) {
    clear_error();
    if (!params || !labels || !ws) return set_error(FHTDP_EINVAL, "null pointer");
    if (!cnn_dims_ok(n, h, w, bands))
        return set_error(FHTDP_EINVAL, "unsupported CNN shape n=%d h=%d w=%d bands=%d", n, h, w,
                         bands);
    const CnnWs c = cnn_ws(n, h, w);
    if (ws_bytes < c.total)
        return set_error(FHTDP_EWORKSPACE, "CNN workspace needs %zu bytes, got %zu", c.total,
                         ws_bytes);
    const char *P = (const char *)params;
    char *W = (char *)ws;
    const int ho = h / 4, wo = w / 4;
    const long long cnt = (long long)n * ho * wo * kC;
    int st = cuda_status(cudaMemsetAsync(W + c.loss, 0, 4, stream), "cudaMemsetAsync");
    // the head's gradient (mean cross-entropy over images and bands)
    if (!st)
        st = cnn_band_head(W + c.act[kLayers - 1], n, ho, wo, bands, labels,
                           1.0f / (float)(n * bands), W + c.g0, (float *)(W + c.loss), nullptr,
                           stream);
    void *dz = W + c.g0, *dx = W + c.g1;
    for (int l = kLayers - 1; l >= 0 && !st; --l) {
        const LayerOff o = layer_off(l);
        float *dw = (float *)(W + c.grads[l]);
        st = cuda_status(cudaMemsetAsync(dw, 0, ((size_t)taps_rows(l) * kC + kC) * 4, stream),
                         "cudaMemsetAsync");
        const void *xin = l == 0 ? (const void *)(W + c.x0) : (const void *)(W + c.act[l - 1]);
        if (!st)
            st = cnn_wgrad(xin, l == 0 ? 1 : kC, n, ho, wo, kDil[l], dz, dw,
                           dw + (size_t)taps_rows(l) * kC, stream);
        if (l == 0 || st) break;
        // input gradient: the forward of the flipped and transposed weights,
        // then the ReLU of the layer below
        if (!st) st = cnn_flip_transpose(P + o.w16, W + c.wflip, stream);
        if (!st) st = cnn_conv3x3(dz, kC, n, ho, wo, kDil[l], W + c.wflip, nullptr, 0, dx, stream);
        if (!st) st = cnn_relu_backward(W + c.act[l - 1], dx, cnt, stream);
        std::swap(dz, dx);
    }
    if (!st && loss)
        st = cuda_status(cudaMemcpyAsync(loss, W + c.loss, 4, cudaMemcpyDeviceToDevice, stream),
                         "cudaMemcpyAsync");
    return st;
}

int fhtdp_cnn_step(void *params, const void *ws, int n, int h, int w, float lr, int step,
                   cudaStream_t stream) {
    clear_error();
    if (!params || !ws || step < 1 || n < 1) return set_error(FHTDP_EINVAL, "bad arguments");
    const CnnWs c = cnn_ws(n, h, w);
    char *P = (char *)params;
    const char *W = (const char *)ws;
    int st = FHTDP_OK;
    for (int l = 0; l < kLayers && !st; ++l) {
        const LayerOff o = layer_off(l);
        const int nw = taps_rows(l) * kC;
        const float *g = (const float *)(W + c.grads[l]);
        st = cnn_adam((float *)(P + o.w), (float *)(P + o.mw), (float *)(P + o.vw), g, nw, lr,
                      0.9f, 0.999f, 1e-8f, step, P + o.w16, stream);
        if (!st)
            st = cnn_adam((float *)(P + o.b), (float *)(P + o.mb), (float *)(P + o.vb), g + nw,
                          kC, lr, 0.9f, 0.999f, 1e-8f, step, nullptr, stream);
    }
    return st;
}

int fhtdp_learned_plan_create(const fhtdp_image *images, int count, int window_half,
                              fhtdp_learned_plan **plan_out) {
    clear_error();
    if (!plan_out || !images || count < 1) return set_error(FHTDP_EINVAL, "bad arguments");
    *plan_out = nullptr;
    const fhtdp_image &a = images[0];
    if (a.h < 1 || a.k < 1 || a.h % a.k || a.h / a.k > 128 || window_half < 0)
        return set_error(FHTDP_EINVAL, "learned detection: bands of at most 128 rows");
    for (int i = 0; i < count; ++i) {
        const fhtdp_image &b = images[i];
        if (b.h != a.h || b.w != a.w || b.k != a.k || b.B != a.B || b.pitch != a.w ||
            (const char *)b.img != (const char *)a.img + (size_t)i * a.h * a.w)
            return set_error(FHTDP_EINVAL,
                             "learned detection: images of one shape, stored one after the other "
                             "([count][h][w], pitch w); image %d differs", i);
    }
    if (!cnn_dims_ok(1, a.h, a.w, a.k))
        return set_error(FHTDP_EINVAL, "learned detection: unsupported CNN shape h=%d w=%d k=%d",
                         a.h, a.w, a.k);
    fhtdp_learned_plan *p = new (std::nothrow) fhtdp_learned_plan();
    if (!p) return set_error(FHTDP_EINVAL, "out of host memory");
    p->N = count;
    p->h = a.h;
    p->w = a.w;
    p->k = a.k;
    p->B = a.B;
    p->half = window_half;
    p->io.assign(images, images + count);
    int st = batch_create(images, count, FHTDP_U8, &p->full);
    if (st) {
        delete p;
        return st;
    }
    p->full_bytes = batch_workspace_bytes(p->full);
    // CNN inference in chunks of at most 64 images (two alternating buffers)
    p->chunk = std::min(count, 64);
    p->cws = cnn_ws_infer(p->chunk, a.h, a.w);
    size_t o = 0;
    p->off_full = o;
    o = align256(o + p->full_bytes);
    p->off_pruned = o;
    o = align256(o + p->full_bytes);   // the same shapes: the same layout
    p->off_cnn = o;
    o = align256(o + p->cws.total);
    p->off_pred = o;
    o = align256(o + (size_t)count * a.k * 4);
    p->off_conf = o;
    o = align256(o + (size_t)count * a.k * 4);
    p->off_win = o;
    o = align256(o + (size_t)count * a.k * 8);
    p->off_x = o;
    o = align256(o + (size_t)count * (a.k + 1) * 4);
    p->off_d = o;
    o = align256(o + (size_t)count * a.k * 4);
    p->off_s = o;
    o = align256(o + (size_t)count * 4);
    p->off_fb = o;
    o = align256(o + (size_t)count * 4);
    p->off_out = o;
    o = align256(o + (size_t)count * sizeof(OutPtrs));
    p->total = o;
    *plan_out = p;
    return FHTDP_OK;
}

size_t fhtdp_learned_workspace_bytes(const fhtdp_learned_plan *plan) {
    return plan ? plan->total : 0;
}

int fhtdp_learned_upload(fhtdp_learned_plan *p, void *ws, size_t ws_bytes, cudaStream_t stream) {
    clear_error();
    if (!p || !ws) return set_error(FHTDP_EINVAL, "null plan or workspace");
    if (ws_bytes < p->total)
        return set_error(FHTDP_EWORKSPACE, "learned workspace needs %zu bytes, got %zu", p->total,
                         ws_bytes);
    char *W = (char *)ws;
    // the pruned batch: windows and scratch outputs in this workspace
    std::vector<fhtdp_image> pr(p->io);
    for (int i = 0; i < p->N; ++i) {
        pr[i].x_out = (int32_t *)(W + p->off_x) + (size_t)i * (p->k + 1);
        pr[i].d_out = (int32_t *)(W + p->off_d) + (size_t)i * p->k;
        pr[i].score_out = (int32_t *)(W + p->off_s) + i;
        pr[i].d_window = (const int32_t *)(W + p->off_win) + (size_t)i * p->k * 2;
    }
    if (p->pruned) batch_destroy(p->pruned);
    p->pruned = nullptr;
    int st = batch_create(pr.data(), p->N, FHTDP_U8, &p->pruned);
    if (st) return st;
    if (batch_workspace_bytes(p->pruned) > p->full_bytes)
        return set_error(FHTDP_EWORKSPACE, "pruned batch layout larger than the full one");
    batch_set_enable(p->full, (const int32_t *)(W + p->off_fb));
    st = batch_upload(p->full, W + p->off_full, p->full_bytes, stream);
    if (!st) st = batch_upload(p->pruned, W + p->off_pruned, p->full_bytes, stream);
    if (st) return st;
    std::vector<OutPtrs> outs(p->N);
    for (int i = 0; i < p->N; ++i)
        outs[i] = OutPtrs{p->io[i].x_out, p->io[i].d_out, (int32_t *)p->io[i].score_out};
    st = cuda_status(cudaMemcpyAsync(W + p->off_out, outs.data(), sizeof(OutPtrs) * p->N,
                                     cudaMemcpyHostToDevice, stream),
                     "cudaMemcpyAsync");
    if (!st) st = cuda_status(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    if (!st) p->bound = ws;
    return st;
}

int fhtdp_detect_learned(fhtdp_learned_plan *p, const void *params, float margin,
                         float min_conf, int32_t *used_fallback, void *ws, cudaStream_t stream) {
    clear_error();
    if (!p || !params || !ws) return set_error(FHTDP_EINVAL, "null plan, params or workspace");
    if (ws != p->bound)
        return set_error(FHTDP_EINVAL, "workspace differs from the one given to fhtdp_learned_upload");
    char *W = (char *)ws;
    const int n = p->h / p->k;
    int32_t *pred = (int32_t *)(W + p->off_pred);
    float *conf = (float *)(W + p->off_conf);
    int32_t *win = (int32_t *)(W + p->off_win);
    int st = FHTDP_OK;
    // 1. the proposal: predicted bins per band, in chunks of images
    const uint8_t *img0 = (const uint8_t *)p->io[0].img;
    for (int c0 = 0; c0 < p->N && !st; c0 += p->chunk) {
        const int cn = std::min(p->chunk, p->N - c0);
        st = forward((const char *)params, img0 + (size_t)c0 * p->h * p->w, cn, p->h, p->w, p->k,
                     W + p->off_cnn, p->cws, pred + (size_t)c0 * p->k, conf + (size_t)c0 * p->k,
                     false, stream);
    }
    // 2. the windows and the pruned DP
    if (!st) st = cnn_bin_windows(pred, p->N * p->k, n, p->half, win, stream);
    if (!st) st = batch_run(p->pruned, W + p->off_pruned, stream);
    // 3. the fallback decision, the full DP of the images that need it (the
    //    others' items are skipped) and the pruned results of the rest
    if (!st) {
        decide_kernel<<<(p->N + 255) / 256, 256, 0, stream>>>(
            p->N, p->k, n, p->h, margin, min_conf, (const int32_t *)(W + p->off_x),
            (const int32_t *)(W + p->off_d), (const int32_t *)(W + p->off_s), win, conf,
            (int32_t *)(W + p->off_fb), used_fallback);
        st = launched("decide_kernel");
    }
    if (!st) st = batch_run(p->full, W + p->off_full, stream);
    if (!st) {
        merge_kernel<<<p->N, 64, 0, stream>>>(p->N, p->k, (const int32_t *)(W + p->off_fb),
                                              (const int32_t *)(W + p->off_x),
                                              (const int32_t *)(W + p->off_d),
                                              (const int32_t *)(W + p->off_s),
                                              (const OutPtrs *)(W + p->off_out));
        st = launched("merge_kernel");
    }
    return st;
}

int fhtdp_learned_status(const fhtdp_learned_plan *p, const void *ws, cudaStream_t stream) {
    clear_error();
    if (!p || !ws) return set_error(FHTDP_EINVAL, "null plan or workspace");
    const char *W = (const char *)ws;
    int st = engine_status(W + p->off_pruned, stream);
    if (!st) st = engine_status(W + p->off_full, stream);
    return st;
}

void fhtdp_learned_plan_destroy(fhtdp_learned_plan *plan) { delete plan; }

}  // extern "C"
