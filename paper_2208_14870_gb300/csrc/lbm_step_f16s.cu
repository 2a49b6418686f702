// Kernels and launchers for the LBM_F16S population storage.
#include "lbm_ops.cuh"

namespace lbm {
template struct Ops<S_F16S>;

cudaError_t step2_f16s(const StepParams& a, const Coef<float>& c, bool gen, bool check,
                       int check_blocks, cudaStream_t st) {
    return launch_step2<S_F16S>(a, c, gen, check, check_blocks, st);
}

cudaError_t step3_f16s(const StepParams& a, const Coef<float>& c, bool gen, bool check,
                      int check_blocks, cudaStream_t st) {
    return launch_step3<S_F16S>(a, c, gen, check, check_blocks, st);
}
}  // namespace lbm
