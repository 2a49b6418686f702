// lbm_noalloc.cu -- lbm_step_checked_noalloc: one residual-checked
// stream-collide step on caller-owned device buffers, for callers that may
// not allocate device memory.
//
// Who needs this: code that runs inside a host application which owns all of
// the device memory through its own pool and does not let plug-ins call
// cudaMalloc, and latency-critical loops that cannot pay for cudaMalloc /
// cudaFree (which may synchronise the whole device).  Such callers already
// hold the populations, the force, the displacement snapshot and the result
// buffer; the only extra memory the residual reduction needs -- one slot of
// partial sums per block and a completion counter -- lives here, in a static
// device array that every GPU loading the library keeps until the process
// exits.
//
// The kernel is the library's persistent residual-check step (k_step with
// CHECK = true); only where its scratch comes from differs.
#include <cmath>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"

using namespace lbm;

namespace {

// Scratch of the residual reduction: LBM_NOALLOC_MAX_BLOCKS slots of kRes
// doubles (one per block of the launch) followed by the completion counter.
constexpr int kCounterOffset = LBM_NOALLOC_MAX_BLOCKS * kRes;  // in doubles
static __device__ __align__(256) double g_noalloc_scratch[kCounterOffset + 32];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};   // device address, per device
int g_resident[kMaxDevices][2][2] = {};           // resident check blocks [dtype F64/F32][V>1]

// Once per device, with that device current: the device address of the
// static scratch array (its host-side name is not a device address).
int scratch_for_device(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return LBM_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<double*>(p);
        int sms = 1;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
        // resident blocks of each check kernel, each query on its own (one
        // block per SM where a query fails; its error is cleared so that the
        // launch check below does not report it)
        auto resident = [&](auto kernel) {
            int b = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kThreads, 0) != cudaSuccess) {
                cudaGetLastError();
                b = 0;
            }
            return sms * (b > 0 ? b : 1);
        };
        g_resident[dev][0][0] = resident(k_step<S_F64, 1, false, true>);
        g_resident[dev][0][1] = resident(k_step<S_F64, 2, false, true>);
        g_resident[dev][1][0] = resident(k_step<S_F32, 1, false, true>);
        g_resident[dev][1][1] = resident(k_step<S_F32, 4, false, true>);
    }
    *out = g_scratch_ptr[dev];
    return LBM_OK;
}

template <typename T>
Coef<T> standard_coef(double lambda, double mu) {
    // Table 1 with theta = 1/3 and w_12 = w_21 = w_22 = 1; Eq. relaxation_rate.
    const double theta = 1.0 / 3.0, K = lambda + mu;
    const double w11 = 1.0 / (mu / theta + 0.5);
    const double ws = 1.0 / (2.0 * K / (1.0 + theta) + 0.5);
    const double wd = 1.0 / (2.0 * mu / (1.0 - theta) + 0.5);
    Coef<T> c{};
    c.q11 = T(0.25 * (1.0 - w11));   // quarter form of collide
    c.qs = T(0.25 * (1.0 - ws));
    c.qd = T(0.25 * (1.0 - wd));
    c.qw12t = T(0.25 * theta);
    c.q12 = T(0.0);
    c.qw21t = T(0.25 * theta);
    c.q21 = T(0.0);
    c.q22 = T(0.0);
    c.qtheta = T(0.25 * theta);
    c.theta = T(theta);
    c.b11 = T(1.0 - 0.5 * w11);
    c.bs = T(1.0 - 0.5 * ws);
    c.bd = T(1.0 - 0.5 * wd);
    return c;
}

}  // namespace

extern "C" int lbm_step_checked_noalloc(int nx, int ny, double lambda, double mu, int dtype,
                                        const void* f_src, void* f_dst, const void* gx,
                                        const void* gy, void* snapshot, double* result,
                                        int grid_blocks, void* stream) {
    if (nx < 1 || ny < 1 || (int64_t)nx * ny > (int64_t)1 << 31)
        return LBM_ERR_ARG;
    if (dtype != LBM_F64 && dtype != LBM_F32)
        return LBM_ERR_ARG;
    if (!std::isfinite(lambda) || !std::isfinite(mu) || !(mu > 0.0) || !(lambda + mu > 0.0))
        return LBM_ERR_ARG;
    if (!f_src || !f_dst || !gx || !gy || !snapshot || !result)
        return LBM_ERR_ARG;
    if (f_src == f_dst)
        return LBM_ERR_ARG;
    if (grid_blocks < 0 || grid_blocks > LBM_NOALLOC_MAX_BLOCKS)
        return LBM_ERR_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_ARG;
    double* scratch = nullptr;
    int rc = scratch_for_device(dev, &scratch);
    if (rc) return rc;

    const int V = dtype == LBM_F64 ? (nx >= 64 ? 2 : 1) : (nx >= 128 ? 4 : 1);
    const int64_t tiles = step_tiles(nx, ny, V);
    int64_t blocks = grid_blocks > 0 ? grid_blocks : g_resident[dev][dtype == LBM_F64 ? 0 : 1][V > 1 ? 1 : 0];
    if (blocks > LBM_NOALLOC_MAX_BLOCKS) blocks = LBM_NOALLOC_MAX_BLOCKS;
    if (blocks > tiles) blocks = tiles;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kCounterOffset);
    // The counter must start at zero; a completed launch leaves it at zero,
    // but clear it anyway so a launch that never ran to its end cannot leak.
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return LBM_ERR_CUDA;

    StepParams a{};
    a.nx = nx;
    a.ny = ny;
    a.plane = (int64_t)nx * ny;
    a.src = f_src;
    a.dst = f_dst;
    a.gx = gx;
    a.gy = gy;
    a.snap = snapshot;
    a.partials = scratch;
    a.counter = counter;
    a.result = result;
    const dim3 block(32, BY);
    const unsigned int grid = (unsigned int)blocks;
    if (dtype == LBM_F64) {
        const Coef<double> c = standard_coef<double>(lambda, mu);
        if (V == 1) k_step<S_F64, 1, false, true><<<grid, block, 0, st>>>(a, c);
        else k_step<S_F64, 2, false, true><<<grid, block, 0, st>>>(a, c);
    } else {
        const Coef<float> c = standard_coef<float>(lambda, mu);
        if (V == 1) k_step<S_F32, 1, false, true><<<grid, block, 0, st>>>(a, c);
        else k_step<S_F32, 4, false, true><<<grid, block, 0, st>>>(a, c);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    return LBM_OK;
}
