// Small helper kernels of the force upload and of the FP16-shifted storage.
#include "lbm_kernels.cuh"

namespace lbm {

__global__ void k_absmax(const double* gx, const double* gy, int64_t n,
                         unsigned long long* out, unsigned int* bad) {
    double m = 0.0;
    unsigned int b = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double a = gx[i], c = gy[i];
        if (!(isfinite(a) && isfinite(c))) b = 1;
        m = fmax(m, fmax(fabs(a), fabs(c)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        b |= __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(m));
        if (b) atomicOr(bad, 1u);
    }
}

__global__ void k_rescale_half(__half* h, int64_t count, float factor) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        h[i] = __float2half_rn(__half2float(h[i]) * factor);
}

}  // namespace lbm
