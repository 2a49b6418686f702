// Kernels and launchers for the LBM_F16S population storage.
#include "lbm_ops.cuh"

namespace lbm {
template struct Ops<S_F16S>;
}  // namespace lbm
