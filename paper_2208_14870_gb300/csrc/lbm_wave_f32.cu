// Wavefront kernels (k_wave, three or four steps per launch) for the LBM_F32
// population storage; a translation unit of their own so that they compile in
// parallel with the other kernels.
#include "lbm_ops.cuh"

namespace lbm {
cudaError_t wave_f32(const StepParams& a, const Coef<float>& c, bool gen, int T, bool check, int seg,
                     cudaStream_t st) {
    return launch_wave<S_F32>(a, c, gen, T, check, seg, st);
}
}  // namespace lbm
