// Kernels and launchers for the LBM_F32 population storage.
#include "lbm_ops.cuh"

namespace lbm {
template struct Ops<S_F32>;
}  // namespace lbm
