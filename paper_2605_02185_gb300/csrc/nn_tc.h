// nn_tc.h -- tcgen05 / TMA convolution kernels of the warm-start network
// (nn_tc.cu), called by the C ABI in nn_kernels.cu.
#pragma once

#include <cuda_runtime.h>

namespace gbnn_tc {

constexpr int kNotEligible = 1;  // shape or alignment the tensor-core kernels do not take

// y = act(conv3x3(x, w) + bias) on the tensor cores (arguments as
// gbnn_conv3x3_fwd).  0 on success, kNotEligible (nothing launched), or -2
// for a CUDA error.
int conv_fwd(const void *x, int xs, const void *w, const float *bias, void *y, int ys, const void *mask, int ms, int N,
             int H, int W, int cin, int cout, int relu, cudaStream_t st);

// gw += dL/dw (and gb += dL/db if gb) on the tensor cores (arguments as
// gbnn_conv3x3_wgrad).  0, kNotEligible (nothing launched) or -2.
int conv_wgrad(const void *x, int xs, const void *gy, int gs, float *gw, float *gb, int N, int H, int W, int cin,
               int cout, int splits, cudaStream_t st);

// Device status word of the tensor-core kernels (1: a bounded wait gave
// up), optionally cleared; -2 if it cannot be read.
int status(int reset);

}  // namespace gbnn_tc
