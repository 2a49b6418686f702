// Kernels and launchers for the LBM_F64 population storage.
#include "lbm_ops.cuh"

namespace lbm {
template struct Ops<S_F64>;
}  // namespace lbm
