// lbm_k_f16sr.cu -- step, init, force, fields and mass kernels for IEEE-half
// storage with stochastic rounding (half_sr).
#include "../../include/gblbm.h"
#include "lbm_kernels.cuh"

namespace gblbm {
const KernelOps *ops_f16sr() { return Launch<half_sr>::table(); }

// The stochastic rounding of the store on its own, for a unit test: value
// x[i] with salt[i] -> the stored 16-bit pattern.
__global__ void round_probe_kernel(int bf16, const float *__restrict__ x, const uint32_t *__restrict__ salt,
                                   uint16_t *__restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    // salt[i] plays the node seed, direction 0
    if (bf16) {
      const bf16_sr r = Store<bf16_sr>::st_at(x[i], salt[i], 0);
      out[i] = __bfloat16_as_ushort(r.v);
    } else {
      const half_sr r = Store<half_sr>::st_at(x[i], salt[i], 0);
      out[i] = __half_as_ushort(r.v);
    }
  }
}
}  // namespace gblbm

extern "C" int lbm_probe_stochastic_round(int storage, const float *x, const uint32_t *salt, uint16_t *out, int64_t n,
                                          void *stream) {
  if (!x || !salt || !out || n <= 0 || (storage != LBM_F16_SR && storage != LBM_BF16_SR)) return LBM_ERR_ARG;
  const long long blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  gblbm::round_probe_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(storage == LBM_BF16_SR, x, salt, out,
                                                                          (long long)n);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
