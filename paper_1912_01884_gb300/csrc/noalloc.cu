// fhtdp_detect_polyline_noalloc: the single-image detection of
// fhtdp_detect_polyline for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: hosts that own and hand out all device
// memory themselves (plugins, fixed-budget services), and real-time loops in
// which an allocation, which may synchronise the device, is not allowed.  This
// entry point takes its scratch from a fixed array that the library itself
// declares, so the caller passes only the image and the outputs.
#include <mutex>

#include "common.cuh"
#include "engine.cuh"

namespace fhtdp {
namespace {

constexpr size_t kNoallocScratchBytes = FHTDP_NOALLOC_SCRATCH_BYTES;

// The built-in scratch.  Every GPU on which this module is loaded holds it
// until the process exits.  In host code its name is only a stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current).
int scratch_on_current_device(void **out) {
    int dev = 0;
    int st = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (st) return st;
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(FHTDP_EINVAL, "device %d beyond the %d supported", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        st = cuda_status(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
        if (st) return st;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return FHTDP_OK;
}

}  // namespace
}  // namespace fhtdp

using namespace fhtdp;

extern "C" int fhtdp_detect_polyline_noalloc(const void *img, int dtype, int h, int w, int pitch,
                                             int k, int B, int32_t *x_out, int32_t *d_out,
                                             void *score_out, cudaStream_t stream) {
    clear_error();
    Shape s;
    if (dtype != FHTDP_U8 && dtype != FHTDP_I32 && dtype != FHTDP_F32)
        return set_error(FHTDP_EINVAL, "unknown dtype %d", dtype);
    if (!make_shape(h, w, k, &s))
        return set_error(FHTDP_EINVAL, "invalid shape h=%d w=%d k=%d", h, w, k);
    if (pitch < w) return set_error(FHTDP_EINVAL, "pitch %d < w %d", pitch, w);
    if (B < 0) return set_error(FHTDP_EINVAL, "bend limit B=%d < 0", B);
    if (!img || !x_out || !d_out || !score_out)
        return set_error(FHTDP_EINVAL, "null image or output pointer");
    const size_t need = engine_workspace_bytes(dtype, s, B);
    if (need > kNoallocScratchBytes)
        return set_error(FHTDP_EWORKSPACE,
                         "this image needs %zu bytes of scratch; the built-in scratch of "
                         "fhtdp_detect_polyline_noalloc holds %zu bytes (use "
                         "fhtdp_detect_polyline with a caller workspace)",
                         need, kNoallocScratchBytes);
    void *ws = nullptr;
    int st = scratch_on_current_device(&ws);
    if (st) return st;
    return engine_detect(img, dtype, pitch, s, B, x_out, d_out, score_out, ws,
                         kNoallocScratchBytes, stream);
}

// The status word of the last fhtdp_detect_polyline_noalloc run sits in the
// control block at the start of the built-in scratch, as it does at the start
// of a caller workspace; reading it waits for `stream`.
extern "C" int fhtdp_detect_polyline_noalloc_status(cudaStream_t stream) {
    clear_error();
    void *ws = nullptr;
    int st = scratch_on_current_device(&ws);
    if (st) return st;
    return engine_status(ws, stream);
}
