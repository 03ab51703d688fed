// lbm_k_bf16.cu -- step, init, force, fields and mass kernels for __nv_bfloat16 storage.
#include "lbm_kernels.cuh"

namespace gblbm {
const KernelOps *ops_bf16() { return Launch<__nv_bfloat16>::table(); }
}  // namespace gblbm
