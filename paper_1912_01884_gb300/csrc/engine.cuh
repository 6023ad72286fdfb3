// The fused detection engine (band FHT + bend-limited DP + read-back).
#pragma once

#include "common.cuh"

namespace fhtdp {

size_t engine_workspace_bytes(int dtype, const Shape &s, int B);
int engine_detect(const void *img, int dtype, int pitch, const Shape &s, int B, int32_t *x_out,
                  int32_t *d_out, void *score_out, void *ws, size_t ws_bytes, cudaStream_t stream);

}  // namespace fhtdp
