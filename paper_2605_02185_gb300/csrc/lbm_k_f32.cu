// lbm_k_f32.cu -- step, init, force, fields and mass kernels for float storage.
#include "../../include/gblbm.h"
#include "lbm_kernels.cuh"

namespace gblbm {
const KernelOps *ops_f32() { return Launch<float>::table(); }

// The collisions' -1/rho on its own, in the one-node float lane and the
// packed pair lane, for a unit test against the correctly rounded quotient.
__global__ void neg_recip_probe_kernel(const float *__restrict__ x, float *__restrict__ y1, float *__restrict__ y2,
                                       long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; 2 * i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long a = 2 * i, b = a + 1 < n ? a + 1 : a;
    y1[a] = neg_recip(LF{x[a]}).v;
    if (b != a) y1[b] = neg_recip(LF{x[b]}).v;
    const LF2 r = neg_recip(LF2{make_float2(x[a], x[b])});
    y2[a] = r.v.x;
    if (b != a) y2[b] = r.v.y;
  }
}
}  // namespace gblbm

extern "C" int lbm_probe_neg_recip(const float *x, float *y_single, float *y_pair, int64_t n, void *stream) {
  if (!x || !y_single || !y_pair || n <= 0) return LBM_ERR_ARG;
  const long long pairs = (n + 1) / 2;
  const long long blocks = (pairs + 255) / 256 < 4096 ? (pairs + 255) / 256 : 4096;
  gblbm::neg_recip_probe_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(x, y_single, y_pair, (long long)n);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
