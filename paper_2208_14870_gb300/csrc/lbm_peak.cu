// lbm_peak.cu -- measured FP64 instruction throughput of the device, the
// denominator of the FP64 storage path's roofline.  That path is bound by
// the FP64 pipe, not by HBM: GB300 issues FP64 arithmetic at a small fraction
// of its FP32 rate, so the roofline needs the device's own figure rather than
// a nominal one.  No counterpart in the paper (a measurement utility).
#include <cuda_runtime.h>

#include <string>

#include "../../include/lbm.h"

namespace lbm {
int set_last_error(int code, const std::string& msg);
}

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread
constexpr int kPeakThreads = 256;

// kChains dependent DFMA chains per thread, `iters` links each; the sum is
// stored so that the compiler keeps every chain.  x -> a x + b with a < 1
// keeps the values bounded.
__global__ void __launch_bounds__(kPeakThreads) k_fp64_fma(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int lbm_fp64_fma_rate(double* ginst_per_s) {
    if (!ginst_per_s) return lbm::set_last_error(LBM_ERR_ARG, "lbm_fp64_fma_rate: null pointer");
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, kPeakThreads, 0) != cudaSuccess)
        return lbm::set_last_error(LBM_ERR_CUDA, "lbm_fp64_fma_rate: device query failed");
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = 1 << 13;
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    int rc = LBM_OK;
    float ms = 0.0f;
    if (cudaMalloc(&out, sizeof(double) * grid * kPeakThreads) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = lbm::set_last_error(LBM_ERR_CUDA, "lbm_fp64_fma_rate: setup failed");
    } else {
        // one warm-up launch, then five timed back to back
        k_fp64_fma<<<grid, kPeakThreads, 0, st>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 5; ++r) k_fp64_fma<<<grid, kPeakThreads, 0, st>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f))
            rc = lbm::set_last_error(LBM_ERR_CUDA, "lbm_fp64_fma_rate: timing failed");
        else
            *ginst_per_s = 5.0 * grid * kPeakThreads * (double)iters * kChains / (ms * 1e-3) / 1e9;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    return rc;
}
