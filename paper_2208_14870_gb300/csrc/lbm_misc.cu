// Small helper kernels of the force upload and of the FP16-shifted storage.
#include "lbm_kernels.cuh"

namespace lbm {

__global__ void k_scale_float(float* v, int64_t count, float factor) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        v[i] *= factor;
}

__global__ void k_rescale_half(__half* h, int64_t count, float factor) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        h[i] = __float2half_rn(__half2float(h[i]) * factor);
}

}  // namespace lbm

namespace lbm {

// Higher-order force correction (Sec. 4, Eqs. force_correction_x/y) in
// lattice units:
//   gx' = gx - (D1 dxx gx + D2 dxy gy + D3 dyy gx)
//   gy' = gy - (D3 dxx gy + D2 dxy gx + D1 dyy gy)
// with periodic central differences per node spacing,
//   dxx g = g(x+1) - 2 g(x) + g(x-1),  dxy g = (g(+,+) - g(+,-) - g(-,+) + g(-,-)) / 4.
__global__ void __launch_bounds__(kFinishThreads) k_residual_finish(const double* partials, int64_t nblocks,
                                                                     double* result) {
    __shared__ double sh[kRes][kFinishThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double w[kRes] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int64_t b = tid;
    // four partial sets in flight per thread
    for (; b + 3 * kFinishThreads < nblocks; b += 4 * kFinishThreads) {
        double q[4][kRes];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kRes; ++k) q[u][k] = partials[(b + u * kFinishThreads) * kRes + k];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            w[0] = fmax(w[0], q[u][0]);
            w[1] = fmax(w[1], q[u][1]);
            w[2] += q[u][2];
            w[3] += q[u][3];
            w[4] = fmax(w[4], q[u][4]);
        }
    }
    for (; b < nblocks; b += kFinishThreads) {
        const double* p = partials + b * kRes;
        w[0] = fmax(w[0], p[0]);
        w[1] = fmax(w[1], p[1]);
        w[2] += p[2];
        w[3] += p[3];
        w[4] = fmax(w[4], p[4]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        w[0] = fmax(w[0], __shfl_xor_sync(0xffffffffu, w[0], o));
        w[1] = fmax(w[1], __shfl_xor_sync(0xffffffffu, w[1], o));
        w[2] += __shfl_xor_sync(0xffffffffu, w[2], o);
        w[3] += __shfl_xor_sync(0xffffffffu, w[3], o);
        w[4] = fmax(w[4], __shfl_xor_sync(0xffffffffu, w[4], o));
    }
    if (lane == 0)
        for (int k = 0; k < kRes; ++k) sh[k][warp] = w[k];
    __syncthreads();
    if (tid == 0) {
        double r[kRes] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < kFinishThreads / 32; ++i) {
            r[0] = fmax(r[0], sh[0][i]);
            r[1] = fmax(r[1], sh[1][i]);
            r[2] += sh[2][i];
            r[3] += sh[3][i];
            r[4] = fmax(r[4], sh[4][i]);
        }
        for (int k = 0; k < kRes; ++k) result[k] = r[k];
    }
}

__global__ void k_force_correct(const double* gx, const double* gy, double* ox, double* oy, int nx,
                                int ny, double d1, double d2, double d3) {
    const int64_t n = (int64_t)nx * ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / nx), x = (int)(i - (int64_t)y * nx);
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x + 1 == nx ? 0 : x + 1;
        const int ym = y == 0 ? ny - 1 : y - 1, yp = y + 1 == ny ? 0 : y + 1;
        const int64_t r0 = (int64_t)y * nx, rm = (int64_t)ym * nx, rp = (int64_t)yp * nx;
        const double gxc = gx[r0 + x], gyc = gy[r0 + x];
        const double gx_xx = gx[r0 + xp] - 2.0 * gxc + gx[r0 + xm];
        const double gx_yy = gx[rp + x] - 2.0 * gxc + gx[rm + x];
        const double gy_xx = gy[r0 + xp] - 2.0 * gyc + gy[r0 + xm];
        const double gy_yy = gy[rp + x] - 2.0 * gyc + gy[rm + x];
        const double gx_xy = 0.25 * (gx[rp + xp] - gx[rm + xp] - gx[rp + xm] + gx[rm + xm]);
        const double gy_xy = 0.25 * (gy[rp + xp] - gy[rm + xp] - gy[rp + xm] + gy[rm + xm]);
        ox[r0 + x] = gxc - (d1 * gx_xx + d2 * gy_xy + d3 * gx_yy);
        oy[r0 + x] = gyc - (d3 * gy_xx + d2 * gx_xy + d1 * gy_yy);
    }
}

}  // namespace lbm
