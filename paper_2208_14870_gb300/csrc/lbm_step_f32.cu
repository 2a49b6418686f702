// Kernels and launchers for the LBM_F32 population storage, including the
// two-steps-per-launch kernel.
#include <mutex>

#include "lbm_ops.cuh"

namespace lbm {
template struct Ops<S_F32>;

namespace {
// The two-step kernels use more than 48 KB of dynamic shared memory, which
// each device must allow once per kernel.
cudaError_t t2_allow_smem() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    e = cudaFuncSetAttribute(k_step2<false, false>, at, kT2Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2<false, true>, at, kT2Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2<true, false>, at, kT2Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2<true, true>, at, kT2Smem);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}
}  // namespace

cudaError_t step2_f32(const StepParams& a, const Coef<float>& c, bool gen, bool check,
                      int check_blocks, cudaStream_t st) {
    if (!step2_fits(a.nx, a.ny)) return cudaErrorInvalidValue;
    cudaError_t e = t2_allow_smem();
    if (e != cudaSuccess) return e;
    const int64_t tiles = step2_tiles(a.nx, a.ny);
    const unsigned int grid = (unsigned int)(check ? (tiles < check_blocks ? tiles : check_blocks) : tiles);
    const dim3 block(kT2Threads);
    if (gen) {
        if (check) k_step2<true, true><<<grid, block, kT2Smem, st>>>(a, c);
        else k_step2<true, false><<<grid, block, kT2Smem, st>>>(a, c);
    } else {
        if (check) k_step2<false, true><<<grid, block, kT2Smem, st>>>(a, c);
        else k_step2<false, false><<<grid, block, kT2Smem, st>>>(a, c);
    }
    return cudaGetLastError();
}

}  // namespace lbm
