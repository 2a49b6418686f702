// lbm_arena.cu -- the persistent chunk kernel of the packed lattice arena
// (see lbm_arena.cuh), one instantiation per storage type (FP32, FP16-shifted)
// and tile width.
#include "lbm_arena.cuh"

namespace lbm {

namespace cg = cooperative_groups;

template <int S, int V, bool CHECK>
__device__ __forceinline__ void arena_tile(const BatchArgs& A, const BatchProb& P, int tile,
                                           int s, ResAcc<S>& acc) {
    StepParams a{};
    const int64_t n = (int64_t)P.nx * P.ny;
    a.nx = P.nx;
    a.ny = P.ny;
    a.plane = n;
    const int src = (P.parity + s) & 1;
    char* ps = src ? A.pop1 : A.pop0;
    char* pd = src ? A.pop0 : A.pop1;
    a.src = ps + P.pop_off;
    a.dst = pd + P.pop_off;
    if (S == S_F16S) {
        char* cs = src ? A.car1 : A.car0;
        char* cd = src ? A.car0 : A.car1;
        a.csrc = reinterpret_cast<const float*>(cs + P.car_off);
        a.cdst = reinterpret_cast<float*>(cd + P.car_off);
        a.hscale = P.hscale;
        a.hinv = P.hinv;
    }
    float* fsb = reinterpret_cast<float*>(A.fs + P.fs_off);
    a.gx = fsb;
    a.gy = fsb + n;
    a.snap = fsb + 2 * n;
    Coef<float> c{};
    c.q11 = P.q11;
    c.qs = P.qs;
    c.qd = P.qd;
    c.qtheta = P.qtheta;
    c.theta = P.theta;
    const int ntx = (P.nx + 32 * V - 1) / (32 * V);
    const int ty = tile / ntx, tx = tile - ty * ntx;
    step_tile<S, V, false, CHECK>(a, c, tx, ty, acc);
}

// Block reduction of one tile's residual partials (converted to FP64 per
// thread) into the problem's FP64 accumulator (maxima through the bit
// patterns of non-negative doubles).
template <int S>
__device__ __forceinline__ void tile_to_problem(const ResAcc<S>& acc, double* dst,
                                                double (&red)[kRes][kThreads / 32]) {
    const int tid = threadIdx.y * 32 + threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double v[kRes];
    res_to_double<S>(acc, v);
    warp_reduce_res(v);
    if (lane == 0)
        for (int k = 0; k < kRes; ++k) red[k][warp] = v[k];
    __syncthreads();
    if (tid == 0) {
        double m0 = 0.0, m1 = 0.0, s2 = 0.0, s3 = 0.0, b = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            m0 = fmax(m0, red[0][w]);
            m1 = fmax(m1, red[1][w]);
            s2 += red[2][w];
            s3 += red[3][w];
            b = fmax(b, red[4][w]);
        }
        unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
        atomicMax(d + 0, (unsigned long long)__double_as_longlong(m0));
        atomicMax(d + 1, (unsigned long long)__double_as_longlong(m1));
        atomicAdd(dst + 2, s2);
        atomicAdd(dst + 3, s3);
        atomicMax(d + 4, (unsigned long long)__double_as_longlong(b));
    }
    __syncthreads();
}

template <int S, int V>
__global__ void __launch_bounds__(kThreads, 2) k_arena_chunk(const BatchArgs A) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double red[kRes][kThreads / 32];
    const int ntiles = *A.ntiles;
    for (int s = 0; s < A.nsteps; ++s) {
        const bool last = (s == A.nsteps - 1);
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const uint2 tl = A.tiles[t];
            const BatchProb P = A.probs[tl.x];
            const bool check = last && P.check;  // uniform over the block
            ResAcc<S> acc;
            if (!check) {
                arena_tile<S, V, false>(A, P, (int)tl.y, s, acc);
            } else {
                arena_tile<S, V, true>(A, P, (int)tl.y, s, acc);
                tile_to_problem<S>(acc, A.acc + (int64_t)tl.x * kRes, red);
            }
        }
        if (s + 1 < A.nsteps) grid.sync();
    }
}

// One tile of two steps (k_step2's tile) of problem P; s counts step pairs.
template <int S, bool CHECK>
__device__ __forceinline__ void arena_tile2(const BatchArgs& A, const BatchProb& P, int tile, int s,
                                            float* sm, ResAcc<S>& acc) {
    StepParams a{};
    const int64_t n = (int64_t)P.nx * P.ny;
    a.nx = P.nx;
    a.ny = P.ny;
    a.plane = n;
    const int src = (P.parity + s) & 1;
    a.src = (src ? A.pop1 : A.pop0) + P.pop_off;
    a.dst = (src ? A.pop0 : A.pop1) + P.pop_off;
    if (S == S_F16S) {
        a.csrc = reinterpret_cast<const float*>((src ? A.car1 : A.car0) + P.car_off);
        a.cdst = reinterpret_cast<float*>((src ? A.car0 : A.car1) + P.car_off);
        a.hscale = P.hscale;
        a.hinv = P.hinv;
    }
    float* fsb = reinterpret_cast<float*>(A.fs + P.fs_off);
    a.gx = fsb;
    a.gy = fsb + n;
    a.snap = fsb + 2 * n;
    Coef<float> c{};
    c.q11 = P.q11;
    c.qs = P.qs;
    c.qd = P.qd;
    c.qtheta = P.qtheta;
    c.theta = P.theta;
    const int ntx = (P.nx + kT2OX - 1) / kT2OX;
    const int ty = tile / ntx, tx = tile - ty * ntx;
    step2_tile<S, false, CHECK, true>(a, c, sm, tx, ty, acc);
}

// The chunk with two steps per tile visit and one grid barrier per pair of
// steps (nsteps even); the residual check rides on the second step of the
// chunk's last pair.
template <int S>
__global__ void __launch_bounds__(kT2Threads, 2) k_arena_chunk2(const BatchArgs A) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ float t2_smem[];
    __shared__ double red[kRes][kThreads / 32];
    const int ntiles = *A.ntiles;
    const int npairs = A.nsteps / 2;
    for (int s = 0; s < npairs; ++s) {
        const bool last = (s == npairs - 1);
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const uint2 tl = A.tiles[t];
            const BatchProb P = A.probs[tl.x];
            const bool check = last && P.check;  // uniform over the block
            ResAcc<S> acc;
            if (!check) {
                arena_tile2<S, false>(A, P, (int)tl.y, s, t2_smem, acc);
            } else {
                arena_tile2<S, true>(A, P, (int)tl.y, s, t2_smem, acc);
                tile_to_problem<S>(acc, A.acc + (int64_t)tl.x * kRes, red);
            }
            __syncthreads();   // the slots are reused by the block's next tile
        }
        if (s + 1 < npairs) grid.sync();
    }
}

// One wavefront item of a wide problem: strip and P.seg-row segment `item`,
// the four steps of pass q (the buffers swap once per pass).
template <int S, bool CHECK>
__device__ __forceinline__ void arena_wave_item(const BatchArgs& A, const BatchProb& P, int item, int q,
                                                float* sm, ResAcc<S>& acc) {
    StepParams a{};
    const int64_t n = (int64_t)P.nx * P.ny;
    a.nx = P.nx;
    a.ny = P.ny;
    a.plane = n;
    const int src = (P.parity + q) & 1;
    a.src = (src ? A.pop1 : A.pop0) + P.pop_off;
    a.dst = (src ? A.pop0 : A.pop1) + P.pop_off;
    if (S == S_F16S) {
        a.csrc = reinterpret_cast<const float*>((src ? A.car1 : A.car0) + P.car_off);
        a.cdst = reinterpret_cast<float*>((src ? A.car0 : A.car1) + P.car_off);
        a.hscale = P.hscale;
        a.hinv = P.hinv;
    }
    float* fsb = reinterpret_cast<float*>(A.fs + P.fs_off);
    a.gx = fsb;
    a.gy = fsb + n;
    a.snap = fsb + 2 * n;
    Coef<float> c{};
    c.q11 = P.q11;
    c.qs = P.qs;
    c.qd = P.qd;
    c.qtheta = P.qtheta;
    c.theta = P.theta;
    const int nstrips = (P.nx + wv_ox<4>() - 1) / wv_ox<4>();
    const int strip = item % nstrips, y0 = (item / nstrips) * P.seg;
    wave_block<S, false, 4, CHECK, int>(a, c, sm, strip, y0, min(P.seg, P.ny - y0), acc);
}

// The chunk of the wavefront schedule: nsteps / 4 passes of four steps.  In
// phase 0 of a pass every listed item is visited once -- a wavefront item
// advances its part of a wide problem by four steps, a two-step tile its part
// of a narrow problem by two -- and in phase 1 the two-step tiles (the list's
// tail, from *nwide) once more.  Blocks take items in list order from an
// atomic counter per phase (the heavy wavefront items first), and the grid
// synchronises between phases.  The residual check rides on the last step of
// the chunk: level 4 of the wavefront items, the second step of the phase-1
// tiles of the last pass.
template <int S>
__global__ void __launch_bounds__(kWvW, 2) k_arena_wave(const BatchArgs A) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ float wsm[];   // wavefront rings, or the two-step slot array
    __shared__ double red[kRes][kThreads / 32];
    __shared__ int next;
    const int ntiles = *A.ntiles, nwide = *A.nwide;
    const int npass = A.nsteps / 4;
    for (int q = 0; q < npass; ++q) {
        const bool last = q == npass - 1;
        for (int phase = 0; phase < 2; ++phase) {
            const int begin = phase == 0 ? 0 : nwide;
            int* ctr = A.counters + 2 * q + phase;
            for (;;) {
                if (threadIdx.x == 0) next = begin + atomicAdd(ctr, 1);
                __syncthreads();
                const int t = next;
                __syncthreads();   // `next` is rewritten for the following item
                if (t >= ntiles) break;
                const uint2 tl = A.tiles[t];
                const BatchProb P = A.probs[tl.x];
                ResAcc<S> acc;
                if (t < nwide) {
                    const bool check = last && P.check;   // uniform over the block
                    if (check) {
                        arena_wave_item<S, true>(A, P, (int)tl.y, q, wsm, acc);
                        tile_to_problem<S>(acc, A.acc + (int64_t)tl.x * kRes, red);
                    } else {
                        arena_wave_item<S, false>(A, P, (int)tl.y, q, wsm, acc);
                    }
                } else {
                    const bool check = last && phase == 1 && P.check;
                    if (check) {
                        arena_tile2<S, true>(A, P, (int)tl.y, 2 * q + phase, wsm, acc);
                        tile_to_problem<S>(acc, A.acc + (int64_t)tl.x * kRes, red);
                    } else {
                        arena_tile2<S, false>(A, P, (int)tl.y, 2 * q + phase, wsm, acc);
                    }
                }
                __syncthreads();   // the shared memory is reused by the next item
            }
            if (!(last && phase == 1)) grid.sync();
        }
    }
}

template <int S>
static cudaError_t wave_arena_allow_smem() {
    return cudaFuncSetAttribute(k_arena_wave<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, wv_smem<S, 4>());
}

template <int S>
static cudaError_t launch_wave_chunk(const BatchArgs& a, int grid, cudaStream_t st) {
    if (a.nsteps % 4) return cudaErrorInvalidValue;
    cudaError_t e = wave_arena_allow_smem<S>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kWvW);
    cfg.dynamicSmemBytes = wv_smem<S, 4>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_arena_wave<S>, a);
}

template <int S>
static cudaError_t t2_arena_allow_smem() {
    return cudaFuncSetAttribute(k_arena_chunk2<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, kT2Smem);
}

template <int S>
static cudaError_t launch_two_step(const BatchArgs& a, int grid, cudaStream_t st) {
    if (a.nsteps % 2) return cudaErrorInvalidValue;
    cudaError_t e = t2_arena_allow_smem<S>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kT2Threads);
    cfg.dynamicSmemBytes = kT2Smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_arena_chunk2<S>, a);
}

template <int S, int V>
static cudaError_t launch_v(const BatchArgs& a, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(32, BY);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_arena_chunk<S, V>, a);
}

cudaError_t launch_arena_chunk(int dtype, int V, const BatchArgs& a, int grid, cudaStream_t st) {
    if (V == kTileWave)
        return dtype == S_F16S ? launch_wave_chunk<S_F16S>(a, grid, st) : launch_wave_chunk<S_F32>(a, grid, st);
    if (V == kTileTwoStep)
        return dtype == S_F16S ? launch_two_step<S_F16S>(a, grid, st) : launch_two_step<S_F32>(a, grid, st);
    if (dtype == S_F16S) {
        switch (V) {
            case 1: return launch_v<S_F16S, 1>(a, grid, st);
            case 2: return launch_v<S_F16S, 2>(a, grid, st);
            case 4: return launch_v<S_F16S, 4>(a, grid, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (V) {
        case 1: return launch_v<S_F32, 1>(a, grid, st);
        case 2: return launch_v<S_F32, 2>(a, grid, st);
        case 4: return launch_v<S_F32, 4>(a, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int S, int V>
static int occ() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_arena_chunk<S, V>, kThreads, 0);
    return b;
}

template <int S>
static int occ2() {
    if (t2_arena_allow_smem<S>() != cudaSuccess) return 0;
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_arena_chunk2<S>, kT2Threads, kT2Smem);
    return b;
}

template <int S>
static int occw() {
    if (wave_arena_allow_smem<S>() != cudaSuccess) return 0;
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_arena_wave<S>, kWvW, wv_smem<S, 4>());
    return b;
}

int arena_occupancy(int dtype, int V) {
    if (V == kTileWave) return dtype == S_F16S ? occw<S_F16S>() : occw<S_F32>();
    if (V == kTileTwoStep) return dtype == S_F16S ? occ2<S_F16S>() : occ2<S_F32>();
    if (dtype == S_F16S) return V == 1 ? occ<S_F16S, 1>() : V == 2 ? occ<S_F16S, 2>() : occ<S_F16S, 4>();
    return V == 1 ? occ<S_F32, 1>() : V == 2 ? occ<S_F32, 2>() : occ<S_F32, 4>();
}

}  // namespace lbm
