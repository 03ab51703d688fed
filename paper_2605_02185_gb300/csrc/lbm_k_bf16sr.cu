// lbm_k_bf16sr.cu -- step, init, force, fields and mass kernels for bfloat16
// storage with stochastic rounding (bf16_sr).
#include "lbm_kernels.cuh"

namespace gblbm {
const KernelOps *ops_bf16sr() { return Launch<bf16_sr>::table(); }
}  // namespace gblbm
