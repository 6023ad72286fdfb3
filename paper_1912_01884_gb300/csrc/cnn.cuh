// Kernels of the learned window proposal (cnn.cu).
#pragma once

#include "common.cuh"

namespace fhtdp {

bool cnn_shape_ok(int H, int W, int dil);
int cnn_downsample4(const uint8_t *img, int N, int H, int W, void *out, cudaStream_t stream);
int cnn_conv3x3(const void *X, int cin, int N, int H, int W, int dil, const void *Wt,
                const float *bias, int relu, void *Y, cudaStream_t stream);
int cnn_relu_backward(const void *Y, void *dY, long long count, cudaStream_t stream);
int cnn_flip_transpose(const void *Wt, void *Wf, cudaStream_t stream);
int cnn_wgrad(const void *X, int cin, int N, int H, int W, int dil, const void *dZ, float *dW,
              float *db, cudaStream_t stream);
int cnn_band_head(const void *L, int N, int H, int W, int bands, const int32_t *labels,
                  float scale, void *dL, float *loss, int32_t *pred, cudaStream_t stream,
                  float *conf = nullptr);
int cnn_he_init(float *w, int rows, int cols, int zero_from, float std, unsigned long long seed,
                cudaStream_t stream);
int cnn_adam(float *p, float *m, float *v, const float *g, int count, float lr, float b1,
             float b2, float eps, int t, void *wb, cudaStream_t stream);
int cnn_to_bf16(const float *src, void *dst, int count, cudaStream_t stream);
// The 32-channel layers on tcgen05 (conv_tc.cu); cnn_tc_status reads (and
// with `clear` resets) their device status, synchronising.
int cnn_conv3x3_tc(const void *X, int N, int H, int W, int dil, const void *Wt,
                   const float *bias, int relu, void *Y, cudaStream_t stream);
int cnn_wgrad_tc(const void *X, int N, int H, int W, int dil, const void *dZ, float *dW,
                 float *db, cudaStream_t stream);
int cnn_tc_status(int clear);
int cnn_bin_windows(const int32_t *pred, int count, int n, int margin, int32_t *win,
                    cudaStream_t stream);

}  // namespace fhtdp
