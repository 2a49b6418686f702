// Kernels and launchers for the LBM_F32 population storage.
#include "lbm_ops.cuh"

namespace lbm {
template struct Ops<S_F32>;

cudaError_t step2_f32(const StepParams& a, const Coef<float>& c, bool gen, bool check,
                      int check_blocks, cudaStream_t st) {
    return launch_step2<S_F32>(a, c, gen, check, check_blocks, st);
}

cudaError_t step3_f32(const StepParams& a, const Coef<float>& c, bool gen, bool check,
                      int check_blocks, cudaStream_t st) {
    return launch_step3<S_F32>(a, c, gen, check, check_blocks, st);
}
}  // namespace lbm
