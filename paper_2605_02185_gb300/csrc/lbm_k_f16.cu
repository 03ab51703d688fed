// lbm_k_f16.cu -- step, init, force, fields and mass kernels for __half storage.
#include "lbm_kernels.cuh"

namespace gblbm {
const KernelOps *ops_f16() { return Launch<__half>::table(); }
}  // namespace gblbm
