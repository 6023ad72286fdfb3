// The fused detection engine (band FHT + bend-limited DP + read-back).
#pragma once

#include "common.cuh"

namespace fhtdp {

struct BatchPlan;

size_t engine_workspace_bytes(int dtype, const Shape &s, int B);
int engine_status(const void *ws, cudaStream_t stream);
int batch_create(const fhtdp_image *images, int count, int dtype, BatchPlan **out);
size_t batch_workspace_bytes(const BatchPlan *plan);
long long batch_items(const BatchPlan *plan);
int batch_upload(BatchPlan *plan, void *ws, size_t ws_bytes, cudaStream_t stream);
int batch_run(const BatchPlan *plan, void *ws, cudaStream_t stream);
int batch_autotune(BatchPlan *plan, void *ws, int reps, cudaStream_t stream, long long *chosen);
void batch_choice(const BatchPlan *plan, int n, int *mode, long long *target, int *tile,
                  int *depth);
int batch_configure(BatchPlan *plan, void *ws, int n, int tile, int depth, cudaStream_t stream);
void batch_destroy(BatchPlan *plan);
void debug_inject(int band, int tile, long long wait_cycles);
void batch_set_enable(BatchPlan *plan, const int32_t *enable);
int batch_separate_count(const BatchPlan *plan);
int batch_angle(BatchPlan *plan, double gamma);
int engine_detect(const void *img, int dtype, int pitch, const Shape &s, int B, int32_t *x_out,
                  int32_t *d_out, void *score_out, void *ws, size_t ws_bytes, cudaStream_t stream,
                  const PointMask *pm = nullptr);
bool engine_takes_point(int dtype, const Shape &s, int j = 1);
int batch_points(BatchPlan *plan, void *ws, const int32_t *points, cudaStream_t stream);
int engine_detect_table(const void *img, int dtype, int pitch, const Shape &s,
                        const WindowTable &t, int32_t *x_out, int32_t *d_out, void *score_out,
                        void *ws, cudaStream_t stream);

}  // namespace fhtdp
