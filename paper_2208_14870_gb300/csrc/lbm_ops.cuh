// lbm_ops.cuh -- launchers of the per-storage kernels; included by exactly one
// translation unit per storage type (lbm_step_f64.cu, lbm_step_f32.cu,
// lbm_step_f16s.cu), which instantiates Ops<S> for its type.
#pragma once

#include <mutex>

#include "lbm_kernels.cuh"

namespace lbm {

// The two-step kernels use more than 48 KB of dynamic shared memory, which
// each device must allow once per kernel.
template <int S>
static cudaError_t t2_allow_smem() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    e = cudaFuncSetAttribute(k_step2<S, false, false, false>, at, kT2Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2<S, false, true, false>, at, kT2Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2<S, true, false, false>, at, kT2Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2<S, true, true, false>, at, kT2Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2<S, false, false, true>, at, kT2Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2<S, false, true, true>, at, kT2Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2<S, true, false, true>, at, kT2Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2<S, true, true, true>, at, kT2Smem);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

template <int S>
static cudaError_t t3_allow_smem() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    e = cudaFuncSetAttribute(k_step3<S, false, false, false>, at, kT3Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step3<S, true, false, false>, at, kT3Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step3<S, false, false, true>, at, kT3Smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step3<S, true, false, true>, at, kT3Smem);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

// Three fused plain steps, one block per tile.  (The library puts residual
// checks on two-step launches; a checked three-step launch is not offered.)
template <int S>
static cudaError_t launch_step3(const StepParams& a, const Coef<float>& c, bool gen, bool check,
                                int check_blocks, cudaStream_t st) {
    (void)check_blocks;
    if (check) return cudaErrorNotSupported;
    cudaError_t e = t3_allow_smem<S>();
    if (e != cudaSuccess) return e;
    const unsigned int grid = (unsigned int)step3_tiles(a.nx, a.ny);
    const dim3 block(kT2Threads);
    const bool any = !step3_fits(a.nx, a.ny);   // lattice smaller than the slot array
    if (any) {
        if (gen) k_step3<S, true, false, true><<<grid, block, kT3Smem, st>>>(a, c);
        else k_step3<S, false, false, true><<<grid, block, kT3Smem, st>>>(a, c);
    } else {
        if (gen) k_step3<S, true, false, false><<<grid, block, kT3Smem, st>>>(a, c);
        else k_step3<S, false, false, false><<<grid, block, kT3Smem, st>>>(a, c);
    }
    return cudaGetLastError();
}

// One wavefront kernel: its dynamic shared memory (above 48 KB) is allowed
// once per device, then it is launched.
template <int S, bool GEN, int T, bool CHECK, typename I>
static cudaError_t launch_wave_k(const StepParams& a, const Coef<float>& c, int seg, unsigned int grid,
                                 cudaStream_t st) {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!done[dev]) {
            e = cudaFuncSetAttribute(k_wave<S, GEN, T, CHECK, I>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     wv_smem<S, T>());
            if (e != cudaSuccess) return e;
            done[dev] = true;
        }
    }
    k_wave<S, GEN, T, CHECK, I><<<grid, kWvW, wv_smem<S, T>(), st>>>(a, c, seg);
    return cudaGetLastError();
}

template <int S, bool GEN, int T, bool CHECK>
static cudaError_t launch_wave_i(const StepParams& a, const Coef<float>& c, int seg, unsigned int grid,
                                 cudaStream_t st) {
    // 32-bit in-plane offsets while a plane has fewer than 2^31 nodes
    if ((int64_t)a.nx * a.ny < (int64_t(1) << 31)) return launch_wave_k<S, GEN, T, CHECK, int>(a, c, seg, grid, st);
    return launch_wave_k<S, GEN, T, CHECK, int64_t>(a, c, seg, grid, st);
}

// T = 3 or 4 fused steps on the wavefront schedule: one block per strip and
// segment of seg output rows (the caller checks wave_fits).  check (T = 4
// only): the last step is the residual-check step, one FP64 partial set per
// block in StepParams::partials (wave_blocks<4> of them).
template <int S>
static cudaError_t launch_wave(const StepParams& a, const Coef<float>& c, bool gen, int T, bool check,
                               int seg, cudaStream_t st) {
    if ((T != 3 && T != 4) || seg < 1 || !wave_fits(a.nx, a.ny) || (check && T != 4))
        return cudaErrorInvalidValue;
    const int64_t blocks = T == 3 ? wave_blocks<3>(a.nx, a.ny, seg) : wave_blocks<4>(a.nx, a.ny, seg);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned int grid = (unsigned int)blocks;
    if (check)
        return gen ? launch_wave_i<S, true, 4, true>(a, c, seg, grid, st)
                   : launch_wave_i<S, false, 4, true>(a, c, seg, grid, st);
    if (T == 3)
        return gen ? launch_wave_i<S, true, 3, false>(a, c, seg, grid, st)
                   : launch_wave_i<S, false, 3, false>(a, c, seg, grid, st);
    return gen ? launch_wave_i<S, true, 4, false>(a, c, seg, grid, st)
               : launch_wave_i<S, false, 4, false>(a, c, seg, grid, st);
}

// Two fused steps: one block per tile (check: up to check_blocks blocks).
template <int S>
static cudaError_t launch_step2(const StepParams& a, const Coef<float>& c, bool gen, bool check,
                                int check_blocks, cudaStream_t st) {
    cudaError_t e = t2_allow_smem<S>();
    if (e != cudaSuccess) return e;
    const int64_t tiles = step2_tiles(a.nx, a.ny);
    const unsigned int grid = (unsigned int)(check ? (tiles < check_blocks ? tiles : check_blocks) : tiles);
    const dim3 block(kT2Threads);
    if (!step2_fits(a.nx, a.ny)) {   // lattice smaller than the slot array
        if (gen) {
            if (check) k_step2<S, true, true, true><<<grid, block, kT2Smem, st>>>(a, c);
            else k_step2<S, true, false, true><<<grid, block, kT2Smem, st>>>(a, c);
        } else {
            if (check) k_step2<S, false, true, true><<<grid, block, kT2Smem, st>>>(a, c);
            else k_step2<S, false, false, true><<<grid, block, kT2Smem, st>>>(a, c);
        }
    } else if (gen) {
        if (check) k_step2<S, true, true, false><<<grid, block, kT2Smem, st>>>(a, c);
        else k_step2<S, true, false, false><<<grid, block, kT2Smem, st>>>(a, c);
    } else {
        if (check) k_step2<S, false, true, false><<<grid, block, kT2Smem, st>>>(a, c);
        else k_step2<S, false, false, false><<<grid, block, kT2Smem, st>>>(a, c);
    }
    return cudaGetLastError();
}


template <int S, int V>
static void launch_step_v(const StepParams& a, const Coef<typename StoreT<S>::T>& c, bool gen,
                          bool check, int check_blocks, cudaStream_t st) {
    const dim3 block(32, BY);
    const int64_t tiles = step_tiles(a.nx, a.ny, V);
    const unsigned int grid = (unsigned int)(check ? (tiles < check_blocks ? tiles : check_blocks)
                                                   : tiles);
    if (gen) {
        if (check) k_step<S, V, true, true><<<grid, block, 0, st>>>(a, c);
        else k_step<S, V, true, false><<<grid, block, 0, st>>>(a, c);
    } else {
        if (check) k_step<S, V, false, true><<<grid, block, 0, st>>>(a, c);
        else k_step<S, V, false, false><<<grid, block, 0, st>>>(a, c);
    }
}

template <int S>
cudaError_t Ops<S>::step(const StepParams& a, const Coef<T>& c, int V, bool gen, bool check,
                         int check_blocks, cudaStream_t st) {
    if (V == 1) launch_step_v<S, 1>(a, c, gen, check, check_blocks, st);
    else launch_step_v<S, max_vec<S>()>(a, c, gen, check, check_blocks, st);
    return cudaGetLastError();
}

template <int S>
cudaError_t Ops<S>::fields(const StepParams& a, const Coef<double>& c, T theta, const FieldOut& out,
                           cudaStream_t st) {
    k_fields<S><<<step_grid(a.nx, a.ny, 1), dim3(32, BY), 0, st>>>(a, c, theta, out);
    return cudaGetLastError();
}

template <int S>
cudaError_t Ops<S>::export_pop(const StepParams& a, T theta, double* out, cudaStream_t st) {
    k_export<S><<<step_grid(a.nx, a.ny, 1), dim3(32, BY), 0, st>>>(a, theta, out);
    return cudaGetLastError();
}

template <int S>
cudaError_t Ops<S>::import_pop(const StepParams& a, T theta, const double* in, cudaStream_t st) {
    k_import<S><<<step_grid(a.nx, a.ny, 1), dim3(32, BY), 0, st>>>(a, theta, in);
    return cudaGetLastError();
}

}  // namespace lbm
