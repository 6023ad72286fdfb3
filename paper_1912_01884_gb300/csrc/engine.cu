// Detection engine, first version: the level-by-level FHT, the in-place DP
// and the read-back, composed on one stream.
#include "engine.cuh"

namespace fhtdp {

size_t engine_workspace_bytes(int dtype, const Shape &s, int B) {
    (void)dtype;
    (void)B;
    size_t hough = (size_t)s.k * 2 * s.n * s.W * 4;
    return 2 * hough;
}

int engine_detect(const void *img, int dtype, int pitch, const Shape &s, int B, int32_t *x_out,
                  int32_t *d_out, void *score_out, void *ws, size_t ws_bytes, cudaStream_t stream) {
    (void)ws_bytes;
    size_t hough = (size_t)s.k * 2 * s.n * s.W;
    int st;
    if (dtype == FHTDP_F32) {
        float *H = (float *)ws, *tmp = H + hough;
        st = launch_fht_stages<float, float>((const float *)img, pitch, s, H, tmp, stream);
        if (!st) st = launch_dp_inplace<float>(H, s, B, stream);
        if (!st) st = launch_backtrack<float>(H, s, B, x_out, d_out, (float *)score_out, stream);
    } else {
        int32_t *H = (int32_t *)ws, *tmp = H + hough;
        if (dtype == FHTDP_U8)
            st = launch_fht_stages<uint8_t, int32_t>((const uint8_t *)img, pitch, s, H, tmp, stream);
        else
            st = launch_fht_stages<int32_t, int32_t>((const int32_t *)img, pitch, s, H, tmp, stream);
        if (!st) st = launch_dp_inplace<int32_t>(H, s, B, stream);
        if (!st)
            st = launch_backtrack<int32_t>(H, s, B, x_out, d_out, (int32_t *)score_out, stream);
    }
    return st;
}

}  // namespace fhtdp
