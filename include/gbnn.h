/*
 * gbnn.h -- C ABI of the BF16 tensor-core kernels of the warm-start network
 * (a convolutional encoder-decoder that predicts a developed shedding field
 * rho, u, v from the cylinder mask, Re and a shedding phase).  The paper has
 * no counterpart: these kernels serve the learned warm start of the solver.
 *
 * Conventions: activations are DEVICE bfloat16 arrays in NHWC order,
 * element (n, h, w, c) at ((n*H + h)*W + w)*cstride + c, so a kernel can read
 * or write a channel slice of a wider buffer (pass the slice's base pointer
 * and the buffer's cstride).  Convolution weights are DEVICE bfloat16
 * [Cout][3][3][Cin]; biases and gradients of weights are DEVICE float.
 * Every call is asynchronous on `stream` (a cudaStream_t, NULL = default) and
 * returns 0, -1 for invalid arguments (no launch) or -2 for a CUDA error.
 * Channel counts and strides must be multiples of 8 where stated and base
 * pointers 16-byte aligned.
 */
#ifndef GBNN_H
#define GBNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- implementation choice ------------------------------------------------
 * GBNN_IMPL_TCGEN05: the Blackwell tensor-core kernels -- tcgen05.mma with the
 *   accumulator in tensor memory, operands staged by the TMA engine into a
 *   multi-stage shared-memory ring.  The forward (and input-gradient) call
 *   takes them when cin (the convolution's input channels) and cout are
 *   multiples of 32 (cout <= 256, or two equal halves of a multiple of 32 up
 *   to 512), both channel strides are multiples of 8 and x, w, y (and mask)
 *   are 16-byte aligned; the weight-gradient call when cin and cout are
 *   multiples of 32, cout <= 256, strides multiples of 8, x and gy 16-byte
 *   aligned.
 * GBNN_IMPL_MMA_SYNC: the warp-level m16n8k16 kernels (every shape).
 * GBNN_IMPL_AUTO (default): tcgen05 where the shape is taken, else mma.sync.
 * gbnn_set_conv_impl applies to every later convolution call of the process
 * (not thread-safe); with GBNN_IMPL_TCGEN05 a shape it does not take returns
 * -1.  gbnn_status reads (and with reset != 0 clears) the device status word
 * of the tensor-core kernels: 1 if one of their bounded waits (2 s) gave up,
 * 0 otherwise, -2 on a CUDA error; it synchronises with the device. */
#define GBNN_IMPL_AUTO 0
#define GBNN_IMPL_MMA_SYNC 1
#define GBNN_IMPL_TCGEN05 2
int gbnn_set_conv_impl(int impl);
int gbnn_conv_impl(void);
int gbnn_status(int reset);

/* y = act(conv3x3(x, w) + bias), zero padding 1.  cin, x_cstride: multiples
 * of 8; cout, y_cstride even.  bias may be NULL.  relu != 0 applies ReLU.
 * If mask is not NULL the result is zeroed where mask (same pixel and
 * channel, stride mask_cstride) is <= 0 -- the ReLU derivative when this call
 * computes an input gradient. */
int gbnn_conv3x3_fwd(const void *x, int x_cstride, const void *w, const float *bias, void *y, int y_cstride,
                     const void *mask, int mask_cstride, int N, int H, int W, int cin, int cout, int relu,
                     void *stream);

/* wf[c][2-dy][2-dx][o] = w[o][dy][dx][c]: the weights of the input gradient. */
int gbnn_flip_weights(const void *w, void *wf, int cout, int cin, void *stream);

/* gx = dL/dx of y = conv3x3(x, w) given gy = dL/dy and w_flipped from
 * gbnn_flip_weights; optional ReLU-derivative mask as in gbnn_conv3x3_fwd.
 * cout multiple of 8, cin even. */
int gbnn_conv3x3_dgrad(const void *gy, int gy_cstride, const void *w_flipped, void *gx, int gx_cstride,
                       const void *mask, int mask_cstride, int N, int H, int W, int cin, int cout, void *stream);

/* gw[o][dy][dx][c] += sum over pixels of gy[p][o] x[p + (dy-1, dx-1)][c]
 * and, if gb is not NULL, gb[o] += sum_p gy[p][o].  FP32 accumulation with
 * split-K partial sums added atomically (order not fixed).  cin, cout and
 * both strides multiples of 8.  splits <= 0 picks a default. */
int gbnn_conv3x3_wgrad(const void *x, int x_cstride, const void *gy, int gy_cstride, float *gw, float *gb, int N,
                       int H, int W, int cin, int cout, int splits, void *stream);

/* 2x2 average pooling of an H x W input (H, W even) and its gradient:
 * gx (+)= 0.25 gy[parent] (accumulate != 0 adds to gx), zeroed where mask
 * (stride mask_cstride, may be NULL) is <= 0. */
int gbnn_avgpool2(const void *x, int x_cstride, void *y, int y_cstride, int N, int H, int W, int C, void *stream);
int gbnn_avgpool2_bwd(const void *gy, int gy_cstride, void *gx, int gx_cstride, const void *mask, int mask_cstride,
                      int N, int H, int W, int C, int accumulate, void *stream);

/* 2x nearest upsampling of an H x W input and its gradient. */
int gbnn_upsample2(const void *x, int x_cstride, void *y, int y_cstride, int N, int H, int W, int C, void *stream);
int gbnn_upsample2_bwd(const void *gy, int gy_cstride, void *gx, int gx_cstride, int N, int H, int W, int C,
                       void *stream);

/* *loss_sum += sum over P pixels and C channels of weight[p] (pred - target)^2
 * (target: DEVICE float [P][C]; weight: DEVICE float [P] or NULL); if grad is
 * not NULL, grad = 2 weight (pred - target) scale (bfloat16, stride
 * grad_cstride). */
int gbnn_mse(const void *pred, int pred_cstride, const float *target, const float *weight, void *grad,
             int grad_cstride, long long P, int C, float scale, float *loss_sum, void *stream);

/* One Adam step (Kingma and Ba 2015, bias-corrected, step count t >= 1) on
 * FP32 parameters; param_bf16 (may be NULL) receives the bfloat16 copy. */
int gbnn_adam(float *param, const float *grad, float *m, float *v, void *param_bf16, long long n, float lr,
              float beta1, float beta2, float eps, int t, void *stream);

/* Network input of one sample, [H][W][8] bfloat16: solid flag, Re feature,
 * sin(phase), cos(phase), x/W, y/H, cos(k (x - x0) - phase),
 * sin(k (x - x0) - phase) with k = wave_k (radians per node) and
 * x0 = wave_x0 (a travelling-wave basis for the wake).  solid: DEVICE uint8
 * [H][W]. */
int gbnn_encode_input(const uint8_t *solid, float re_feature, float phase, float wave_k, float wave_x0, int H, int W,
                      void *x, void *stream);

/* Training target [P][3] = ((rho - 1)/rho_scale, (u - U)/vel_scale,
 * v/vel_scale) from DEVICE float fields, and per-pixel loss weight (1 on
 * fluid, 0 on solid; may be NULL). */
int gbnn_encode_target(const float *rho, const float *u, const float *v, const uint8_t *solid, long long P, float U,
                       float vel_scale, float rho_scale, float *target, float *weight, void *stream);

/* Inverse map of a network output (bfloat16, channels 0..2) to DEVICE float
 * fields; solid nodes get rho = 1, u = v = 0. */
int gbnn_decode_output(const void *out, int out_cstride, const uint8_t *solid, long long P, float U, float vel_scale,
                       float rho_scale, float *rho, float *u, float *v, void *stream);

/* cudaMemsetAsync(ptr, 0, bytes) on stream. */
int gbnn_fill_zero(void *ptr, size_t bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GBNN_H */
