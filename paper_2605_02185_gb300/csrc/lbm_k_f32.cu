// lbm_k_f32.cu -- step, init, force, fields and mass kernels for float storage.
#include "lbm_kernels.cuh"

namespace gblbm {
const KernelOps *ops_f32() { return Launch<float>::table(); }
}  // namespace gblbm
