// lbm_k_f64.cu -- step, init, force, fields and mass kernels for double storage.
#include "lbm_kernels.cuh"

namespace gblbm {
const KernelOps *ops_f64() { return Launch<double>::table(); }
}  // namespace gblbm
