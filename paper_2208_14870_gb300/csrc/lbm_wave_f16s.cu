// Wavefront kernels (k_wave, three or four steps per launch) for the LBM_F16S
// population storage; a translation unit of their own so that they compile in
// parallel with the other kernels.
#include "lbm_ops.cuh"

namespace lbm {
cudaError_t wave_f16s(const StepParams& a, const Coef<float>& c, bool gen, int T, bool check, int seg,
                      cudaStream_t st) {
    return launch_wave<S_F16S>(a, c, gen, T, check, seg, st);
}
}  // namespace lbm
