// lbm_kernels.cuh -- CUDA kernels of the periodic lattice Boltzmann scheme for
// linear elasticity (arXiv 2208.14870): fused stream-collide step (Algorithm 1)
// with an optional fused steady-state residual, solution recovery (Table 2),
// population import/export and force upload.  Instantiated once per storage
// type by lbm_step_f64.cu, lbm_step_f32.cu and lbm_step_f16s.cu.
//
// Memory layout (structure of arrays): population p of node (x, y) lives at
// base + p*plane + y*nx + x; `plane` >= nx*ny is padded to 256 bytes.  The
// stored state between steps is the post-collision population f*_p(x) of the
// previous step ("pull" scheme): a step gathers f_p(x) = f*_p(x - c_p) with the
// periodic wrap done by index arithmetic (Sec. 5.1), collides, and writes
// f*_p(x) to the other buffer of a ping-pong pair.
//
// Thread mapping: a block of 32 x BY threads covers a tile of 32*V columns by
// BY rows; a thread handles V nodes of one row spaced 32 apart, so each warp
// load or store instruction touches 32 consecutive nodes of one plane.
#pragma once

#include <type_traits>

#include "lbm_core.cuh"

namespace lbm {

// Launch shape (compile-time): rows per block, resident blocks per SM the
// plain step is compiled for, and nodes per thread of the FP16-shifted wide
// variant. The defaults are the fastest of a sweep at 16384^2 on GB300
// (FP32: BY 8, 4 blocks, 4 nodes; FP16S: 4 blocks of 2 nodes beat 3 of 4).
#ifndef LBM_BY
#define LBM_BY 8
#endif
#ifndef LBM_MINB_F32
#define LBM_MINB_F32 4
#endif
#ifndef LBM_MINB_F16S
#define LBM_MINB_F16S 4
#endif
#ifndef LBM_F16S_V
#define LBM_F16S_V 2
#endif
#ifndef LBM_MINB_F64
#define LBM_MINB_F64 3
#endif
constexpr int BY = LBM_BY;         // rows per block (block = 32 x BY threads)

enum Storage { S_F64 = 0, S_F32 = 1, S_F16S = 2 };

// Nodes per thread (spaced 32 apart) of the wide step variant per storage.
template <int S>
constexpr int max_vec() {
    return S == S_F64 ? 2 : (S == S_F16S ? LBM_F16S_V : 4);
}
constexpr int kThreads = 32 * BY;

template <int S> struct StoreT;
// T: collision arithmetic, P: stored population, G: stored force.
template <> struct StoreT<S_F64> { using T = double; using P = double; using G = double; };
template <> struct StoreT<S_F32> { using T = float; using P = float; using G = float; };
template <> struct StoreT<S_F16S> { using T = float; using P = __half; using G = float; };

// Residual partial sums of one block: max|du|, max|u|, sum du^2, sum u^2,
// non-finite flag.
constexpr int kRes = 5;

struct StepParams {
    int nx, ny;
    int64_t plane;          // elements between planes
    const void* src;        // 8 population planes (storage type)
    void* dst;
    const float* csrc;      // F16S: carriers (m*_10, m*_01) interleaved per node (float2)
    float* cdst;
    const void* gx;         // force planes (G)
    const void* gy;
    float hscale;           // F16S: the state's scale 2^e (see store_f16s)
    float hinv;             // 1 / hscale
    void* snap;             // residual: u_x, u_y snapshot, 2 planes of nx*ny (ResSnap)
    double* partials;       // residual: kRes doubles per block
    unsigned int* counter;  // residual: blocks finished, reset by the last block; null:
                            // blocks only write partials (k_residual_finish combines them)
    double* result;         // residual: kRes doubles
};

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// Steady-state residual (Sec. 2.1's stopping test; reading: max and L2 norms
// of u^t - u^(t-w) over a window of w steps).  Each thread keeps partials over
// its nodes -- max|du|, max|u| (over nodes and both components), sum du^2,
// sum u^2 and a non-finite flag -- and the snapshot holds u of the previous
// check, two planes of nx*ny entries:
//   FP64 storage: u from the FP64 collision, FP64 snapshot and partials;
//   FP32 / FP16S: u as an exact FP32 pair from exact_displacement, the
//   snapshot as (hi, lo) pairs (16 bytes per node, like two FP64 planes), and
//   pair partials (about 2^-44 relative), converted to FP64 per thread.
// Warps, blocks and the grid combine the partials in FP64.
template <int S> struct ResSnap { float2 u, v; };          // (hi, lo) per component
template <> struct ResSnap<S_F64> { double u, v; };

template <int S> struct ResAcc {
    float dh = 0.f, dl = 0.f, uh = 0.f, ul = 0.f, d2h = 0.f, d2l = 0.f, u2h = 0.f, u2l = 0.f, bad = 0.f;
};
template <> struct ResAcc<S_F64> {
    double d = 0.0, u = 0.0, d2 = 0.0, u2 = 0.0, bad = 0.0;
};

// max(m, |h + l|) on normalised pairs (|l| <= ulp(h) / 2), lexicographically.
// Once a thread's running maximum is established few nodes reach it, so the
// full comparison sits behind one test of the hi part.
__device__ __forceinline__ void pair_max_abs(float& mh, float& ml, float h, float l) {
    if (fabsf(h) >= mh) {
        if (h < 0.0f) {
            h = -h;
            l = -l;
        }
        if (h > mh || l > ml) {
            mh = h;
            ml = l;
        }
    }
}

// s += (h + l)^2 in pair arithmetic: h*h with its exact FMA error, plus
// 2 h l (l^2 is below 2^-48 h^2 and dropped); the sum stays normalised.
__device__ __forceinline__ void pair_add_square(float& sh, float& sl, float h, float l) {
    const float p = __fmul_rn(h, h);
    const float e = fmaf(2.0f * h, l, fmaf(h, h, -p));
    float t;
    const float s = two_sum(sh, p, t);
    sh = fast_two_sum(s, __fadd_rn(sl, __fadd_rn(t, e)), sl);
}

template <int S>
__device__ __forceinline__ ResSnap<S> snap_load(const StepParams& a, int64_t n, int64_t idx) {
    ResSnap<S> o;
    if constexpr (S == S_F64) {
        const double* sp = static_cast<const double*>(a.snap);
        o.u = sp[idx];
        o.v = sp[n + idx];
    } else {
        const float2* sp = static_cast<const float2*>(a.snap);
        o.u = sp[idx];
        o.v = sp[n + idx];
    }
    return o;
}

// Residual check of one node: compare u^t of the step's input state (pulled
// populations f, force g; FP64 storage: the collision's u, v) with the
// snapshot entry `old` loaded before, store u^t as the new snapshot entry and
// update the thread's partials.
template <int S>
__device__ __forceinline__ void check_node(const StepParams& a, int64_t n, int64_t idx, ResAcc<S>& acc,
                                           const ResSnap<S>& old, const typename StoreT<S>::T f[8],
                                           typename StoreT<S>::T gx, typename StoreT<S>::T gy,
                                           typename StoreT<S>::T u, typename StoreT<S>::T v) {
    if constexpr (S == S_F64) {
        (void)f;
        (void)gx;
        (void)gy;
        double* sp = static_cast<double*>(a.snap);
        sp[idx] = u;
        sp[n + idx] = v;
        const double du = u - old.u, dv = v - old.v;
        acc.d = fmax(acc.d, fmax(fabs(du), fabs(dv)));
        acc.u = fmax(acc.u, fmax(fabs(u), fabs(v)));
        acc.d2 += du * du + dv * dv;
        acc.u2 += u * u + v * v;
        if (!(isfinite(u) && isfinite(v))) acc.bad = 1.0;
    } else {
        (void)u;
        (void)v;
        const float4 w = exact_displacement(f, gx, gy);
        float2* sp = static_cast<float2*>(a.snap);
        sp[idx] = make_float2(w.x, w.y);
        sp[n + idx] = make_float2(w.z, w.w);
        float e, dl;
        // du = u^t - u^(t-w) as a pair: the hi parts' difference exactly,
        // then the lo parts' (both below an ulp of u)
        float dh = two_sum(w.x, -old.u.x, e);
        dh = two_sum(dh, __fadd_rn(e, __fsub_rn(w.y, old.u.y)), dl);
        pair_max_abs(acc.dh, acc.dl, dh, dl);
        pair_add_square(acc.d2h, acc.d2l, dh, dl);
        dh = two_sum(w.z, -old.v.x, e);
        dh = two_sum(dh, __fadd_rn(e, __fsub_rn(w.w, old.v.y)), dl);
        pair_max_abs(acc.dh, acc.dl, dh, dl);
        pair_add_square(acc.d2h, acc.d2l, dh, dl);
        pair_max_abs(acc.uh, acc.ul, w.x, w.y);
        pair_max_abs(acc.uh, acc.ul, w.z, w.w);
        pair_add_square(acc.u2h, acc.u2l, w.x, w.y);
        pair_add_square(acc.u2h, acc.u2l, w.z, w.w);
        if (!(isfinite(w.x) && isfinite(w.z))) acc.bad = 1.0f;
    }
}

// The thread's partials in FP64: [max|du|, max|u|, sum du^2, sum u^2, flag].
template <int S>
__device__ __forceinline__ void res_to_double(const ResAcc<S>& acc, double w[kRes]) {
    if constexpr (S == S_F64) {
        w[0] = acc.d;
        w[1] = acc.u;
        w[2] = acc.d2;
        w[3] = acc.u2;
        w[4] = acc.bad;
    } else {
        w[0] = (double)acc.dh + (double)acc.dl;
        w[1] = (double)acc.uh + (double)acc.ul;
        w[2] = (double)acc.d2h + (double)acc.d2l;
        w[3] = (double)acc.u2h + (double)acc.u2l;
        w[4] = acc.bad;
    }
}

// Warp-level FP64 combination of kRes partials (result in every lane).
__device__ __forceinline__ void warp_reduce_res(double w[kRes]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        w[0] = fmax(w[0], __shfl_xor_sync(0xffffffffu, w[0], o));
        w[1] = fmax(w[1], __shfl_xor_sync(0xffffffffu, w[1], o));
        w[2] += __shfl_xor_sync(0xffffffffu, w[2], o);
        w[3] += __shfl_xor_sync(0xffffffffu, w[3], o);
        w[4] = fmax(w[4], __shfl_xor_sync(0xffffffffu, w[4], o));
    }
}

// Stored values that the pull of one node reads: the 8 populations f*_p(x - c_p)
// as stored (and, FP16S, the carriers of the 8 source nodes).
template <int S> struct Pulled { typename StoreT<S>::P p[8]; };
template <> struct Pulled<S_F16S> { __half p[8]; float2 c[8]; };

// Load the stored values of the pull of node (x, y) (loads only).
// r0, rm, rp: offsets of rows y, y-1, y+1 (wrapped); xm, xp: columns x-1, x+1.
// I: in-plane offset type (int where a plane has fewer than 2^31 nodes).
template <int S, typename I = int64_t>
__device__ __forceinline__ void pull_load(const StepParams& a, I r0, I rm, I rp,
                                          int x, int xm, int xp, Pulled<S>& q) {
    using P = typename StoreT<S>::P;
    const P* s = static_cast<const P*>(a.src);
    const int64_t pl = a.plane;
    const I i0 = r0 + xm, i1 = rm + x, i2 = r0 + xp, i3 = rp + x;
    const I i4 = rm + xm, i5 = rm + xp, i6 = rp + xp, i7 = rp + xm;
    if constexpr (S == S_F16S) {
        // carriers interleaved per node: (m*_10, m*_01) as one float2
        const float2* c = reinterpret_cast<const float2*>(a.csrc);
        q.c[0] = ldg(c + i0);
        q.c[1] = ldg(c + i1);
        q.c[2] = ldg(c + i2);
        q.c[3] = ldg(c + i3);
        q.c[4] = ldg(c + i4);
        q.c[5] = ldg(c + i5);
        q.c[6] = ldg(c + i6);
        q.c[7] = ldg(c + i7);
    }
    q.p[0] = ldg(s + 0 * pl + i0);
    q.p[1] = ldg(s + 1 * pl + i1);
    q.p[2] = ldg(s + 2 * pl + i2);
    q.p[3] = ldg(s + 3 * pl + i3);
    q.p[4] = ldg(s + 4 * pl + i4);
    q.p[5] = ldg(s + 5 * pl + i5);
    q.p[6] = ldg(s + 6 * pl + i6);
    q.p[7] = ldg(s + 7 * pl + i7);
}

// The pre-collision populations f_p(x) from the pulled stored values
// (FP16S: the stored deviation + the equilibrium part of the source carrier,
// both in the state's scaled units; see store_f16s).
template <int S>
__device__ __forceinline__ void pull_decode(const StepParams& a, const Pulled<S>& q,
                                            typename StoreT<S>::T f[8], typename StoreT<S>::T theta) {
    using T = typename StoreT<S>::T;
    if constexpr (S == S_F16S) {
        (void)a;
        const float k1 = 0.5f * (1.0f - theta), k5 = 0.25f * theta;
        f[0] = fmad(k1, q.c[0].x, __half2float(q.p[0]));
        f[1] = fmad(k1, q.c[1].y, __half2float(q.p[1]));
        f[2] = fmad(-k1, q.c[2].x, __half2float(q.p[2]));
        f[3] = fmad(-k1, q.c[3].y, __half2float(q.p[3]));
        f[4] = fmad(k5, q.c[4].x + q.c[4].y, __half2float(q.p[4]));
        f[5] = fmad(k5, q.c[5].y - q.c[5].x, __half2float(q.p[5]));
        f[6] = fmad(-k5, q.c[6].x + q.c[6].y, __half2float(q.p[6]));
        f[7] = fmad(k5, q.c[7].x - q.c[7].y, __half2float(q.p[7]));
    } else {
        (void)a;
        (void)theta;
#pragma unroll
        for (int p = 0; p < 8; ++p) f[p] = T(q.p[p]);
    }
}

// Gather the pre-collision populations of node (x, y): f_p(x) = f*_p(x - c_p).
template <int S>
__device__ __forceinline__ void gather(const StepParams& a, int64_t r0, int64_t rm, int64_t rp,
                                       int x, int xm, int xp, typename StoreT<S>::T f[8],
                                       typename StoreT<S>::T theta) {
    Pulled<S> q;
    pull_load<S>(a, r0, rm, rp, x, xm, xp, q);
    pull_decode<S>(a, q, f, theta);
}

// FP16-shifted store of one node: the deviations N (FP32) are rounded to
// FP16, and the FP32 carriers absorb the first moments of the ROUNDED
// deviations, c10 = m*_10 - m_10(N_rounded), so that the stored state
// N_rounded + E(c) keeps the first moments m*_10, m*_01 exactly (E(c) has
// first moments c, no second moments).  Without this, the rounding of N would
// feed the conserved mean-displacement mode every step and u would drift.
// Scaled units: an FP16S lattice keeps its whole FP32 state -- carriers,
// force, intermediate populations, residual snapshot -- multiplied by its
// power-of-two scale 2^e (StepParams::hscale), chosen so that the deviations
// sit well inside FP16's normal range.  The scale commutes with every
// rounding, so this is the same arithmetic as unscaled values with the FP16
// rounding done on N 2^e, without a multiplication per population in the
// decode and two here; only the recovery, the export, the import and the
// reported norms of u convert.
__device__ __forceinline__ void store_f16s(const StepParams& a, int64_t idx, const float n[8],
                                           float m10s, float m01s) {
    __half* d = static_cast<__half*>(a.dst);
    const int64_t pl = a.plane;
    float r[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const __half h = __float2half_rn(n[p]);
        d[p * pl + idx] = h;
        r[p] = __half2float(h);
    }
    const float e10 = (r[0] - r[2]) + ((r[4] - r[6]) - (r[5] - r[7]));
    const float e01 = (r[1] - r[3]) + ((r[4] - r[6]) + (r[5] - r[7]));
    reinterpret_cast<float2*>(a.cdst)[idx] = make_float2(m10s - e10, m01s - e01);
}

// The values a node stores after its collision (raw moments m, force g; GEN
// as for collide): the eight post-collision populations, or for FP16S the
// eight deviations N and the carriers (c10, c01) = (m*_10, m*_01); u, v
// receive the displacement.  Computed apart from the stores so that kernels
// can run it on every thread and predicate only the stores.
template <int S, bool GEN>
__device__ __forceinline__ void post_state(const Mom<typename StoreT<S>::T>& m, typename StoreT<S>::T gx,
                                           typename StoreT<S>::T gy, const Coef<typename StoreT<S>::T>& c,
                                           typename StoreT<S>::T& u, typename StoreT<S>::T& v,
                                           typename StoreT<S>::T f[8], float& c10, float& c01) {
    using T = typename StoreT<S>::T;
    if constexpr (S == S_F16S) {
        const Mom<T> s = collide<T, GEN>(m, gx, gy, c, u, v);
        populations<!GEN>(deviation_moments(s, c.qtheta), f);
        c10 = s.m10;
        c01 = s.m01;
    } else {
        collide_populations<GEN>(m, gx, gy, c, u, v, f);
        c10 = c01 = 0.0f;
    }
}

// Store the post_state values of node idx.
template <int S>
__device__ __forceinline__ void store_state(const StepParams& a, int64_t idx, const typename StoreT<S>::T f[8],
                                            float c10, float c01) {
    using P = typename StoreT<S>::P;
    if constexpr (S == S_F16S) {
        store_f16s(a, idx, f, c10, c01);
    } else {
        P* d = static_cast<P*>(a.dst);
        const int64_t pl = a.plane;
#pragma unroll
        for (int p = 0; p < 8; ++p) d[p * pl + idx] = P(f[p]);
    }
}

// Collide node idx (raw moments m, force g) and store its post-collision
// state.
template <int S, bool GEN>
__device__ __forceinline__ void scatter_local(const StepParams& a, int64_t idx,
                                              const Mom<typename StoreT<S>::T>& m,
                                              typename StoreT<S>::T gx, typename StoreT<S>::T gy,
                                              const Coef<typename StoreT<S>::T>& c) {
    typename StoreT<S>::T f[8], u, v;
    float c10, c01;
    post_state<S, GEN>(m, gx, gy, c, u, v, f, c10, c01);
    store_state<S>(a, idx, f, c10, c01);
}

// Residual reduction of a block.  Each thread's partials (ResAcc) are
// converted to FP64 and combined across the warp, the block and the grid in
// FP64.  With a counter, the grid-level pass is done by the last block to
// finish (counted with an atomic), which also resets the counter for the next
// check; without one (the library's own check launches) the blocks stop after
// writing their partials and k_residual_finish combines them in a separate
// launch.
template <int S>
__device__ __forceinline__ void residual_reduce(const StepParams& a, const ResAcc<S>& acc) {
    __shared__ double sh[kRes][kThreads / 32];
    __shared__ bool is_last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y) >> 5;
    double v[kRes];
    res_to_double<S>(acc, v);
    warp_reduce_res(v);
    if (lane == 0)
        for (int k = 0; k < kRes; ++k) sh[k][warp] = v[k];
    __syncthreads();
    const unsigned int nblocks = gridDim.x * gridDim.y;
    const unsigned int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (tid == 0) {
        double w[kRes] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < nwarps; ++i) {
            w[0] = fmax(w[0], sh[0][i]);
            w[1] = fmax(w[1], sh[1][i]);
            w[2] += sh[2][i];
            w[3] += sh[3][i];
            w[4] = fmax(w[4], sh[4][i]);
        }
        for (int k = 0; k < kRes; ++k) a.partials[(int64_t)bid * kRes + k] = w[k];
        if (a.counter != nullptr) {
            __threadfence();
            const unsigned int done = atomicAdd(a.counter, 1u);
            is_last = (done == nblocks - 1);
        }
    }
    // Partials only: a later k_residual_finish launch combines them, so the
    // block ends here without a memory fence or a grid counter.
    if (a.counter == nullptr) return;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // (four blocks' partials in flight per thread: the grid may have 10^5 blocks)
    double w[kRes] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const unsigned int nthr = blockDim.x * blockDim.y;
    unsigned int b = tid;
    for (; b + 3 * nthr < nblocks; b += 4 * nthr) {
        double q[4][kRes];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kRes; ++k) q[u][k] = __ldcg(a.partials + (int64_t)(b + u * nthr) * kRes + k);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            w[0] = fmax(w[0], q[u][0]);
            w[1] = fmax(w[1], q[u][1]);
            w[2] += q[u][2];
            w[3] += q[u][3];
            w[4] = fmax(w[4], q[u][4]);
        }
    }
    for (; b < nblocks; b += nthr) {
        const double* p = a.partials + (int64_t)b * kRes;
        w[0] = fmax(w[0], __ldcg(p + 0));
        w[1] = fmax(w[1], __ldcg(p + 1));
        w[2] += __ldcg(p + 2);
        w[3] += __ldcg(p + 3);
        w[4] = fmax(w[4], __ldcg(p + 4));
    }
    warp_reduce_res(w);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < kRes; ++k) sh[k][warp] = w[k];
    __syncthreads();
    if (tid == 0) {
        double r[kRes] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < nwarps; ++i) {
            r[0] = fmax(r[0], sh[0][i]);
            r[1] = fmax(r[1], sh[1][i]);
            r[2] += sh[2][i];
            r[3] += sh[3][i];
            r[4] = fmax(r[4], sh[4][i]);
        }
        for (int k = 0; k < kRes; ++k) a.result[k] = r[k];
        *a.counter = 0u;
        __threadfence();
    }
}

// One pseudo-time step (Algorithm 1) over the whole lattice.
//
// The lattice is cut into tiles of 32*V columns by BY rows; block b handles
// tiles b, b + gridDim.x, ...  The plain step is launched with one block per
// tile.  CHECK adds the steady-state residual: u^t (the displacement of this
// step's input state) is compared with the snapshot taken at the previous
// check, the snapshot is overwritten with u^t, and each block reduces its
// partials once, after all of its tiles (FP64 across warps, blocks and the
// grid).  The library launches it with one block per tile up to
// kMaxCheckBlocks blocks (more tiles per block beyond that).
// One tile of one step: tile (tx, ty) covers columns tx*32V .. tx*32V+32V-1
// and rows ty*BY .. ty*BY+BY-1.  With CHECK the thread's residual partials
// are accumulated into acc.
template <int S, int V, bool GEN, bool CHECK>
__device__ __forceinline__ void step_tile(const StepParams& a,
                                          const Coef<typename StoreT<S>::T>& c, int tx, int ty,
                                          ResAcc<S>& acc) {
    using T = typename StoreT<S>::T;
    using G = typename StoreT<S>::G;
    const int nx = a.nx, ny = a.ny;
    const int y = ty * BY + threadIdx.y;
    const int xb = tx * (32 * V) + threadIdx.x;
    if (y >= ny) return;
    const G* __restrict__ gxp = static_cast<const G*>(a.gx);
    const G* __restrict__ gyp = static_cast<const G*>(a.gy);
    const int64_t n = (int64_t)nx * ny;
    const int ym = wrap_dec(y, ny), yp = wrap_inc(y, ny);
    const int64_t r0 = (int64_t)y * nx, rm = (int64_t)ym * nx, rp = (int64_t)yp * nx;
    // Phase 1: issue every load of the thread's V nodes before any store,
    // so that up to V*10 (V*12 with the snapshot) loads are in flight.
    T f[V][8], gx[V], gy[V];
    ResSnap<S> so[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const int x = xb + 32 * j;
        if (x < nx) {
            gather<S>(a, r0, rm, rp, x, wrap_dec(x, nx), wrap_inc(x, nx), f[j], c.theta);
            gx[j] = T(ldg(gxp + r0 + x));
            gy[j] = T(ldg(gyp + r0 + x));
            if (CHECK) so[j] = snap_load<S>(a, n, r0 + x);
        }
    }
    // Phase 2: collide and store.
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const int x = xb + 32 * j;
        if (x < nx) {
            const int64_t idx = r0 + x;
            const Mom<T> m = moments(f[j]);
            scatter_local<S, GEN>(a, idx, m, gx[j], gy[j], c);
            if (CHECK) {
                T u, v;
                displacement(m, gx[j], gy[j], u, v);
                check_node<S>(a, n, idx, acc, so[j], f[j], gx[j], gy[j], u, v);
            }
        }
    }
}

template <int S, int V, bool GEN, bool CHECK>
__global__ void __launch_bounds__(kThreads, CHECK ? 2 : (S == S_F32 ? LBM_MINB_F32 : (S == S_F16S ? LBM_MINB_F16S : LBM_MINB_F64)))
k_step(const StepParams a, const Coef<typename StoreT<S>::T> c) {
    const int ntx = (a.nx + 32 * V - 1) / (32 * V);
    const int64_t ntiles = (int64_t)ntx * ((a.ny + BY - 1) / BY);
    ResAcc<S> acc;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int ty = (int)(t / ntx), tx = (int)(t - (int64_t)ty * ntx);
        step_tile<S, V, GEN, CHECK>(a, c, tx, ty, acc);
    }
    if (CHECK) residual_reduce<S>(a, acc);
}

// ---------------------------------------------------------------------------
// Two pseudo-time steps per launch, FP32 or FP16-shifted storage (temporal
// blocking).
//
// A block of 256 threads (8 warps) owns one output tile of kT2OX x kT2OY
// nodes (62 x 22) and a slot array of kT2W x kT2H nodes (64 x 24, 48 KB of
// FP32 populations): the tile grown by one node on every side.  Step 1 pulls the stored f*(t) from global memory exactly as
// the single step does, collides every slot and keeps f*(t+1) of all slots in
// shared memory; step 2 pulls f*(t+1) of the tile's nodes from shared memory
// (their pull neighbours are the halo slots), collides again and stores
// f*(t+2) of the tile.  The state crosses HBM once per two steps: per node and
// launch 32 bytes read, 32 written and 8 of force read, i.e. 36 bytes per
// lattice update instead of 72 (FP16-shifted: 28 instead of 56).  Thread
// (lane, warp) owns slot columns lane and lane + 32 and slot rows warp + 8k in
// both steps, so the force it loaded in step 1 serves step 2 from registers.
// The per-node arithmetic is the single step's (gather, collide, populations),
// so with FP32 storage a launch reproduces two single-step launches exactly.
// With FP16-shifted storage the intermediate state f*(t+1) stays in FP32
// (only the state written back is rounded to the storage format), so results
// differ from one step per launch by less than the storage rounding.
//
// Any lattice size works: slot coordinates wrap periodically, and a lattice
// smaller than the slot array appears in it more than once (ANY = true, the
// general wrap; the batched arena uses it for every problem).  A lattice of
// at least kT2W x kT2H (step2_fits) takes the ANY = false kernel, whose wrap
// is one conditional subtraction.  CHECK makes the second step the
// residual-check step of k_step<..., CHECK> (snapshot compared with u^{t+1},
// the second step's input state); its snapshot loads are issued before the
// barrier between the steps.
#ifndef LBM_T2_RPW
#define LBM_T2_RPW 3
#endif
#ifndef LBM_MINB_T2
#define LBM_MINB_T2 3
#endif
#ifndef LBM_MINB_T2_F16S
#define LBM_MINB_T2_F16S 4
#endif
#ifndef LBM_T2_B
#define LBM_T2_B 1
#endif
constexpr int kT2Rows = LBM_T2_RPW;             // slot rows per warp
constexpr int kT2B = LBM_T2_B;                  // slot rows gathered together in step 1
static_assert(kT2Rows % kT2B == 0, "rows per warp must be a multiple of the gather batch");
constexpr int kT2W = 64;                        // slot columns (two per lane)
constexpr int kT2H = 8 * kT2Rows;               // slot rows
constexpr int kT2OX = kT2W - 2, kT2OY = kT2H - 2;
constexpr int kT2Threads = 256;
constexpr int kT2Smem = 8 * kT2H * kT2W * (int)sizeof(float);
static_assert(kT2Threads == kThreads, "residual_reduce sizes its scratch by kThreads");

// Periodic image in [0, n) of a slot coordinate v >= -1.  ANY = false
// needs n at least the slot span (one conditional subtraction); ANY = true
// serves any n (a lattice smaller than the slot array appears in it more
// than once).  The two are separate kernels because the general form costs
// the large-lattice kernel 4-6 % even where it never takes the long path.
template <bool ANY>
__device__ __forceinline__ int wrap_slot(int v, int n) {
    if (v < 0) v += n;
    if (ANY && v < 0) v = v % n + n;   // v >= -2 on a lattice of one node
    if (v >= n) v = (!ANY || v < 2 * n) ? v - n : v % n;
    return v;
}

template <int S, bool GEN, bool CHECK, bool ANY>
__device__ __forceinline__ void step2_tile(const StepParams& a, const Coef<float>& c, float* sm,
                                           int tx, int ty, ResAcc<S>& acc) {
    constexpr int PL = kT2H * kT2W;             // shared-memory plane
    const int nx = a.nx, ny = a.ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = tx * kT2OX - 1, y0 = ty * kT2OY - 1;   // node of slot (0, 0)
    const float* __restrict__ gxp = static_cast<const float*>(a.gx);
    const float* __restrict__ gyp = static_cast<const float*>(a.gy);
    int X[2], XM[2], XP[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int x = wrap_slot<ANY>(x0 + lane + 32 * j, nx);
        X[j] = x;
        XM[j] = wrap_dec(x, nx);
        XP[j] = wrap_inc(x, nx);
    }
    float gx[kT2Rows][2], gy[kT2Rows][2];   // force of the thread's slots
    // Step 1: f*(t+1) of every slot into shared memory.
#pragma unroll
    for (int kb = 0; kb < kT2Rows; kb += kT2B) {
        float f[kT2B][2][8];
#pragma unroll
        for (int b = 0; b < kT2B; ++b) {
            const int k = kb + b;
            const int y = wrap_slot<ANY>(y0 + warp + 8 * k, ny);
            const int64_t r0 = (int64_t)y * nx;
            const int64_t rm = (int64_t)wrap_dec(y, ny) * nx, rp = (int64_t)wrap_inc(y, ny) * nx;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                gather<S>(a, r0, rm, rp, X[j], XM[j], XP[j], f[b][j], c.theta);
                gx[k][j] = ldg(gxp + r0 + X[j]);
                gy[k][j] = ldg(gyp + r0 + X[j]);
            }
        }
#pragma unroll
        for (int b = 0; b < kT2B; ++b) {
            const int k = kb + b, r = warp + 8 * k;
            float* s = sm + r * kT2W + lane;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                float u, v, fs[8];
                collide_populations<GEN>(moments(f[b][j]), gx[k][j], gy[k][j], c, u, v, fs);
#pragma unroll
                for (int p = 0; p < 8; ++p) s[p * PL + 32 * j] = fs[p];
            }
        }
    }
    const int64_t n = (int64_t)nx * ny;
    ResSnap<S> so[kT2Rows][2];
    if (CHECK) {
#pragma unroll
        for (int k = 0; k < kT2Rows; ++k) {
            const int r = warp + 8 * k, y = y0 + r;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int col = lane + 32 * j, x = x0 + col;
                if (r >= 1 && r <= kT2H - 2 && y < ny && col >= 1 && col <= kT2W - 2 && x < nx)
                    so[k][j] = snap_load<S>(a, n, (int64_t)y * nx + x);
            }
        }
    }
    __syncthreads();
    // Step 2: the tile's nodes pull f*(t+1) from shared memory.
#pragma unroll
    for (int k = 0; k < kT2Rows; ++k) {
        const int r = warp + 8 * k;
        const int y = y0 + r;
        if (r < 1 || r > kT2H - 2 || y >= ny) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int col = lane + 32 * j;
            const int x = x0 + col;
            if (col < 1 || col > kT2W - 2 || x >= nx) continue;
            const int64_t idx = (int64_t)y * nx + x;
            const float* s = sm + r * kT2W + col;
            float f[8];
            f[0] = s[0 * PL - 1];               // f_p(x) = f*_p(x - c_p)
            f[1] = s[1 * PL - kT2W];
            f[2] = s[2 * PL + 1];
            f[3] = s[3 * PL + kT2W];
            f[4] = s[4 * PL - kT2W - 1];
            f[5] = s[5 * PL - kT2W + 1];
            f[6] = s[6 * PL + kT2W + 1];
            f[7] = s[7 * PL + kT2W - 1];
            const Mom<float> m = moments(f);
            scatter_local<S, GEN>(a, idx, m, gx[k][j], gy[k][j], c);
            if (CHECK) {
                float u, v;
                displacement(m, gx[k][j], gy[k][j], u, v);
                check_node<S>(a, n, idx, acc, so[k][j], f, gx[k][j], gy[k][j], u, v);
            }
        }
    }
}

#ifndef LBM_MINB_T2_CHECK
#define LBM_MINB_T2_CHECK 3
#endif
template <int S, bool GEN, bool CHECK, bool ANY>
__global__ void __launch_bounds__(kT2Threads,
                                  CHECK ? LBM_MINB_T2_CHECK : (S == S_F16S ? LBM_MINB_T2_F16S : LBM_MINB_T2))
k_step2(const StepParams a, const Coef<float> c) {
    extern __shared__ float t2_smem[];
    const int ntx = (a.nx + kT2OX - 1) / kT2OX;
    const int64_t ntiles = (int64_t)ntx * ((a.ny + kT2OY - 1) / kT2OY);
    ResAcc<S> acc;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int ty = (int)(t / ntx), tx = (int)(t - (int64_t)ty * ntx);
        step2_tile<S, GEN, CHECK, ANY>(a, c, t2_smem, tx, ty, acc);
        if (t + gridDim.x < ntiles) __syncthreads();   // slots are reused by the next tile
    }
    if (CHECK) residual_reduce<S>(a, acc);
}

// ---------------------------------------------------------------------------
// Three pseudo-time steps per launch (FP32 or FP16-shifted storage).
//
// The two-step scheme carried one step further: a block of 256 threads owns an
// output tile of kT3OX x kT3OY nodes (60 x 12) and two shared-memory slot
// arrays A and B of kT3W x kT3H slots (64 x 16, 32 KB each): the tile grown
// by two nodes on every side.  Step 1 pulls f*(t) from global memory and
// writes f*(t+1) of every slot to A; step 2 pulls from A and writes f*(t+2)
// of the slots one node inside the edge to B; step 3 pulls from B and stores
// f*(t+3) of the tile.  Per node and launch the state crosses HBM once: 72 B
// (FP32) or 56 B (FP16S) for three lattice updates.  Thread (lane, warp) owns
// slot columns lane and lane + 32 and rows warp + 8k in all three steps; the
// per-node arithmetic is the single step's, so FP32 results equal three
// single-step launches bit for bit (FP16S keeps the two intermediate states
// in FP32).  CHECK would make the third step the residual-check step; the
// library puts its checks on two-step launches instead, which cost less
// relative to their plain form.  ANY as for k_step2; the library uses the
// ANY = false kernel from kT3W x kT3H nodes up.
#ifndef LBM_T3_RPW
#define LBM_T3_RPW 2
#endif
#ifndef LBM_MINB_T3
#define LBM_MINB_T3 3
#endif
constexpr int kT3Rows = LBM_T3_RPW;             // slot rows per warp
constexpr int kT3W = 64;                        // slot columns (two per lane)
constexpr int kT3H = 8 * kT3Rows;               // slot rows
constexpr int kT3OX = kT3W - 4, kT3OY = kT3H - 4;
constexpr int kT3Smem = 2 * 8 * kT3H * kT3W * (int)sizeof(float);

template <int S, bool GEN, bool CHECK, bool ANY>
__device__ __forceinline__ void step3_tile(const StepParams& a, const Coef<float>& c, float* smA,
                                           int tx, int ty, ResAcc<S>& acc) {
    constexpr int PL = kT3H * kT3W;             // shared-memory plane
    float* smB = smA + 8 * PL;
    const int nx = a.nx, ny = a.ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = tx * kT3OX - 2, y0 = ty * kT3OY - 2;   // node of slot (0, 0)
    const float* __restrict__ gxp = static_cast<const float*>(a.gx);
    const float* __restrict__ gyp = static_cast<const float*>(a.gy);
    int X[2], XM[2], XP[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int x = wrap_slot<ANY>(x0 + lane + 32 * j, nx);
        X[j] = x;
        XM[j] = wrap_dec(x, nx);
        XP[j] = wrap_inc(x, nx);
    }
    float gx[kT3Rows][2], gy[kT3Rows][2];
    // Step 1: f*(t+1) of every slot into A.
#pragma unroll
    for (int k = 0; k < kT3Rows; ++k) {
        const int r = warp + 8 * k;
        const int y = wrap_slot<ANY>(y0 + r, ny);
        const int64_t r0 = (int64_t)y * nx;
        const int64_t rm = (int64_t)wrap_dec(y, ny) * nx, rp = (int64_t)wrap_inc(y, ny) * nx;
        float f[2][8];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            gather<S>(a, r0, rm, rp, X[j], XM[j], XP[j], f[j], c.theta);
            gx[k][j] = ldg(gxp + r0 + X[j]);
            gy[k][j] = ldg(gyp + r0 + X[j]);
        }
        float* s = smA + r * kT3W + lane;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float u, v, fs[8];
            collide_populations<GEN>(moments(f[j]), gx[k][j], gy[k][j], c, u, v, fs);
#pragma unroll
            for (int p = 0; p < 8; ++p) s[p * PL + 32 * j] = fs[p];
        }
    }
    __syncthreads();
    // Step 2: f*(t+2) of the slots one node inside the edge, from A into B.
#pragma unroll
    for (int k = 0; k < kT3Rows; ++k) {
        const int r = warp + 8 * k;
        if (r < 1 || r > kT3H - 2) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int col = lane + 32 * j;
            if (col < 1 || col > kT3W - 2) continue;
            const float* s = smA + r * kT3W + col;
            float f[8];
            f[0] = s[0 * PL - 1];               // f_p(x) = f*_p(x - c_p)
            f[1] = s[1 * PL - kT3W];
            f[2] = s[2 * PL + 1];
            f[3] = s[3 * PL + kT3W];
            f[4] = s[4 * PL - kT3W - 1];
            f[5] = s[5 * PL - kT3W + 1];
            f[6] = s[6 * PL + kT3W + 1];
            f[7] = s[7 * PL + kT3W - 1];
            float u, v, fs[8];
            collide_populations<GEN>(moments(f), gx[k][j], gy[k][j], c, u, v, fs);
            float* d = smB + r * kT3W + col;
#pragma unroll
            for (int p = 0; p < 8; ++p) d[p * PL] = fs[p];
        }
    }
    const int64_t n = (int64_t)nx * ny;
    ResSnap<S> so[kT3Rows][2];
    if (CHECK) {
#pragma unroll
        for (int k = 0; k < kT3Rows; ++k) {
            const int r = warp + 8 * k, y = y0 + r;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int col = lane + 32 * j, x = x0 + col;
                if (r >= 2 && r <= kT3H - 3 && y < ny && col >= 2 && col <= kT3W - 3 && x < nx)
                    so[k][j] = snap_load<S>(a, n, (int64_t)y * nx + x);
            }
        }
    }
    __syncthreads();
    // Step 3: the tile's nodes pull f*(t+2) from B and store f*(t+3).
#pragma unroll
    for (int k = 0; k < kT3Rows; ++k) {
        const int r = warp + 8 * k;
        const int y = y0 + r;
        if (r < 2 || r > kT3H - 3 || y >= ny) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int col = lane + 32 * j;
            const int x = x0 + col;
            if (col < 2 || col > kT3W - 3 || x >= nx) continue;
            const int64_t idx = (int64_t)y * nx + x;
            const float* s = smB + r * kT3W + col;
            float f[8];
            f[0] = s[0 * PL - 1];
            f[1] = s[1 * PL - kT3W];
            f[2] = s[2 * PL + 1];
            f[3] = s[3 * PL + kT3W];
            f[4] = s[4 * PL - kT3W - 1];
            f[5] = s[5 * PL - kT3W + 1];
            f[6] = s[6 * PL + kT3W + 1];
            f[7] = s[7 * PL + kT3W - 1];
            const Mom<float> m = moments(f);
            scatter_local<S, GEN>(a, idx, m, gx[k][j], gy[k][j], c);
            if (CHECK) {
                float u, v;
                displacement(m, gx[k][j], gy[k][j], u, v);
                check_node<S>(a, n, idx, acc, so[k][j], f, gx[k][j], gy[k][j], u, v);
            }
        }
    }
}

template <int S, bool GEN, bool CHECK, bool ANY>
__global__ void __launch_bounds__(kT2Threads, LBM_MINB_T3)
k_step3(const StepParams a, const Coef<float> c) {
    extern __shared__ float t3_smem[];
    const int ntx = (a.nx + kT3OX - 1) / kT3OX;
    const int64_t ntiles = (int64_t)ntx * ((a.ny + kT3OY - 1) / kT3OY);
    ResAcc<S> acc;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int ty = (int)(t / ntx), tx = (int)(t - (int64_t)ty * ntx);
        step3_tile<S, GEN, CHECK, ANY>(a, c, t3_smem, tx, ty, acc);
        if (t + gridDim.x < ntiles) __syncthreads();   // slots are reused by the next tile
    }
    if (CHECK) residual_reduce<S>(a, acc);
}

// ---------------------------------------------------------------------------
// Wavefront schedule of T pseudo-time steps per launch (FP32 or FP16-shifted
// storage; T = 3 or 4).
//
// A block of 32*NW threads owns a strip of W = 32*NW slot columns (thread t
// = column t for the whole launch) and a segment of `seg` output rows, and
// walks down the segment one row per iteration at every step level at once:
// in iteration i, step tau (1..T) updates the row of local index i - 2(tau - 1)
// (local row j is lattice row ybeg + j, ybeg = y0 - (T - 1)), so step tau
// trails step tau - 1 by two rows and only reads rows that step tau - 1
// finished in earlier iterations.  Step 1 pulls f*(t) from global memory,
// steps 2..T-1 pull from and write to rings of kWvD = 4 rows per level in
// shared memory (local row j in ring slot j mod 4), and step T stores
// f*(t+T) of the strip's W - 2(T-1) inner columns to global memory.  One
// block barrier per iteration separates a ring slot's last read from its next
// write.  The halo costs 2(T-1) of W columns and 2(T - tau) extra rows of
// level tau per segment, and a level's ring holds four rows instead of a
// whole tile, so four steps per launch fit.
//
// The vertical movers c_2 = (0, 1) and c_4 = (0, -1) are pulled from the
// thread's own column, so they skip the rings: each level boundary keeps them
// in a per-thread delay line (population 2 of the last three rows produced,
// population 4 of the last one), and the rings hold the six other
// populations.  Step 1 pulls into registers one row ahead of its use (FP32
// with LBM_WV_LA2_F32: two rows) and loads the force two rows ahead (FP16S:
// one row; its pulls carry the FP32 carriers too).
//
// Instruction economy (the kernel issues, it does not wait on HBM): the
// iterations in which every level is active run in groups of four, so every
// ring slot is a compile-time offset from one per-thread address and no
// level tests whether it is active; only the first 3(T-1) and the last few
// iterations of a segment take the general path.  The force of a thread's
// column for the last 2(T-1)+1 rows stays in registers (step tau uses the row
// step 1 loaded 2(tau-1) iterations earlier).  With I = int (lattices below
// 2^31 nodes) global addresses are a 32-bit in-plane offset on a per-plane
// base.
//
// CHECK: step T is the residual-check step (its input state is u^(t+T-1));
// its snapshot loads run one iteration ahead, and the block's partials go to
// StepParams::partials (k_residual_finish combines them).
//
// The per-node arithmetic is the single step's: FP32 results equal T
// single-step launches bit for bit (FP16S keeps the intermediate states in
// FP32).  Lattices from W x 8 nodes up.
#ifndef LBM_WV_NW
#define LBM_WV_NW 8
#endif
// step 1: populations loaded two rows ahead (1) or one (0), per storage type
// (FP16S pulls hold three times the registers; two rows ahead measured 1 %
// slower)
#ifndef LBM_WV_LA2_F32
#define LBM_WV_LA2_F32 1
#endif
#ifndef LBM_WV_LA2_F16S
#define LBM_WV_LA2_F16S 0
#endif
constexpr int kWvNW = LBM_WV_NW;                 // warps per block
constexpr int kWvW = 32 * kWvNW;                 // strip width (slot columns)
constexpr int kWvRow = kWvW + 2;                 // ring row: the strip plus one pad column per side
constexpr int kWvD = 4;                          // ring rows per level
constexpr int kWvRP = 6;                         // populations held in a ring (all but 2 and 4)
constexpr int kWvSegDefault = 256;               // output rows per block segment (default)
template <int S>
__host__ __device__ constexpr bool wv_la2() {
    return S == S_F16S ? LBM_WV_LA2_F16S != 0 : LBM_WV_LA2_F32 != 0;
}
// step 1 collides its row at the start of the iteration (1), so its decoded
// populations die before the other levels run and its load buffers are free
// for the next row, or after the other levels (0), so its loads are issued
// earlier.  Defaults: the faster at 16384^2 on GB300 (FP32 after: 3.34 against
// 3.77 ms per four-step launch; FP16S first: 3.48 against 3.72 ms)
#ifndef LBM_WV_L1FIRST_F32
#define LBM_WV_L1FIRST_F32 0
#endif
#ifndef LBM_WV_L1FIRST_F16S
#define LBM_WV_L1FIRST_F16S 1
#endif
// FP32: step 1's load buffers and the delay lines of population 2 as
// circular buffers of four, indexed by the iteration's phase in its group of
// four (no register copies: 3.31 against 3.35 ms per four-step launch at
// 16384^2 on GB300), or (0) two buffers whose pulls are copied before the
// reload, and delay lines shifted every iteration
#ifndef LBM_WV_CIRC
#define LBM_WV_CIRC 1
#endif
template <int S>
__host__ __device__ constexpr bool wv_l1first() {
    return S == S_F16S ? LBM_WV_L1FIRST_F16S != 0 : LBM_WV_L1FIRST_F32 != 0;
}
static_assert(kWvW <= kThreads, "residual_reduce sizes its scratch by kThreads");
template <int T> __host__ __device__ constexpr int wv_ox() { return kWvW - 2 * (T - 1); }
template <int S, int T> __host__ __device__ constexpr int wv_smem() {
    return (T - 1) * kWvRP * kWvD * kWvRow * (int)sizeof(float);
}
// resident blocks per SM the kernel is compiled for: what 228 KB of shared
// memory per SM allows (1 KB reserved per block), at most LBM_WV_MINB (the
// register budget: 128 registers a thread at two blocks of 256 threads)
#ifndef LBM_WV_MINB
#define LBM_WV_MINB 2
#endif
template <int S, int T> constexpr int wv_minb() {
    return (233472 / (wv_smem<S, T>() + 1024)) < LBM_WV_MINB ? (233472 / (wv_smem<S, T>() + 1024))
                                                             : LBM_WV_MINB;
}

// One block's share of a wavefront launch: strip `strip`, output rows y0 ..
// y0 + rows - 1, T steps; wv_ring is the block's (T-1) rings.  With CHECK the thread's residual partials of
// level T are accumulated into acc.  Called by k_wave (one block per strip
// and segment) and by the batched arena (one call per work item).
template <int S, bool GEN, int T, bool CHECK, typename I, bool CIRC_OK = false>
__device__ __forceinline__ void wave_block(const StepParams& a, const Coef<float>& c, float* wv_ring,
                                           int strip, int y0, int rows, ResAcc<S>& acc) {
    static_assert(T >= 2 && T <= 4, "two to four steps per launch");
    constexpr int W = kWvW, R = kWvRow, OX = wv_ox<T>(), PL = kWvD * kWvRow, RP = kWvRP * PL, D = kWvD - 1;
    constexpr bool PA2 = wv_la2<S>();             // populations two rows ahead
    constexpr bool L1FIRST = wv_l1first<S>();     // step 1 collides before the other levels
    // (CIRC_OK: the single-lattice kernel; the batched arena's kernel, which also
    // holds the two-step tiles, spills more with the larger code and keeps the
    // copies: 2048 problems of sides 32 to 1024 ran at 141 against 165 GLUPS with them)
    constexpr bool CIRC = CIRC_OK && LBM_WV_CIRC != 0 && S == S_F32 && PA2 && !L1FIRST;
    const int nx = a.nx, ny = a.ny;
    const int t = threadIdx.x;
    const int xs = strip * OX - (T - 1) + t;      // lattice column of slot t (unwrapped)
    const int x = wrap_slot<false>(xs, nx);
    const int xm = wrap_dec(x, nx), xp = wrap_inc(x, nx);
    const bool store_ok = t >= T - 1 && t <= W - T && xs < nx;
    const float* __restrict__ gxp = static_cast<const float*>(a.gx);
    const float* __restrict__ gyp = static_cast<const float*>(a.gy);
    const int ybeg = y0 - (T - 1);                // lattice row of local row 0 (level 1)
    const int iters = rows + 3 * (T - 1);
    const int n1 = rows + 2 * (T - 1);            // rows of level 1
    const int64_t n = (int64_t)nx * ny;
    // This thread's column of every ring (slot t sits at padded column t + 1,
    // so the pulls of t - 1 and t + 1 stay inside the row for every thread).
    float* const rt = wv_ring + t + 1;
    // Force of the thread's column in local rows i, i - 1, ..., i - 2(T - 1)
    // (i the iteration): level tau uses entry 2(tau - 1).
    constexpr int NH = 2 * (T - 1) + 1;
    float hx[NH], hy[NH];
#pragma unroll
    for (int k = 0; k < NH; ++k) hx[k] = hy[k] = 0.0f;
    // Delay lines of the vertical movers at the T - 1 level boundaries: v2[r][k]
    // is population 2 (index 1) of the row ring r's producer made k + 1
    // productions ago, v4[r] population 4 (index 3) of its last row.  The
    // consumer (level r + 2) of local row j reads population 2 of row j - 1
    // (made three iterations earlier) and population 4 of row j + 1 (one
    // iteration earlier) before the producer (level r + 1) of the same
    // iteration shifts the line; producers run in consecutive iterations, from
    // three iterations before their consumer's first to one before its last.
    float v2[T - 1][4], v4[T - 1];
#pragma unroll
    for (int r = 0; r < T - 1; ++r) v2[r][0] = v2[r][1] = v2[r][2] = v2[r][3] = v4[r] = 0.0f;
    // Step 1's pulls (one row ahead, PA2: two) and the force (LA2: two rows
    // ahead, else one) in registers.  The row offsets of the next row to load
    // advance one row per load (rows are loaded in order), with the periodic
    // wrap.
    constexpr bool LA2 = S == S_F32 || PA2;
    Pulled<S> q[CIRC ? 4 : (PA2 ? 2 : 1)];
    float qg[LA2 ? 2 : 1][2];
    int ly = wrap_slot<false>(ybeg, ny);          // lattice row of the next population load
    I lr0 = (I)ly * nx, lrm = (I)wrap_dec(ly, ny) * nx, lrp = (I)wrap_inc(ly, ny) * nx;
    int gly = ly;                                 // lattice row of the next force load
    auto advance = [&]() {
        ly = wrap_inc(ly, ny);
        lrm = lr0;
        lr0 = lrp;
        lrp = (I)wrap_inc(ly, ny) * nx;
    };
    auto load_force = [&](int b) {
        const I g = (I)gly * nx + x;
        qg[b][0] = ldg(gxp + g);
        qg[b][1] = ldg(gyp + g);
        gly = wrap_inc(gly, ny);
    };
    auto load1 = [&](int b) {
        pull_load<S, I>(a, lr0, lrm, lrp, x, xm, xp, q[b]);
        advance();
    };
    // Residual check on level T: its snapshot entry is loaded one iteration ahead.
    ResSnap<S> so;
    auto snap_next = [&](int i) {
        so = snap_load<S>(a, n, (int64_t)((I)(ybeg + i - 2 * (T - 1)) * nx + xs));
    };

    // One iteration; FULL: every level active (ring slots fold to constants
    // when i is a compile-time offset from a multiple of four).
    // Halo threads of a level compute values no valid slot reads (their pulls
    // stay inside the padded ring rows), so no level branches per thread; only
    // the stores of level T are predicated.
    auto iter = [&](int i, auto full_c, auto buf_c) {
        constexpr bool FULL = decltype(full_c)::value;
        constexpr int K = decltype(buf_c)::value;   // phase: i mod 4 (CIRC), else i mod 2
        constexpr int b = LA2 ? (K & 1) : 0;        // load buffers of local row i (i mod 2 with
                                                    // two rows ahead, else 0)
        const bool l1 = FULL || i < n1;
#pragma unroll
        for (int k = NH - 1; k > 0; --k) {
            hx[k] = hx[k - 1];
            hy[k] = hy[k - 1];
        }
        hx[0] = qg[b][0];
        hy[0] = qg[b][1];
        // step 1 on local row i: its populations 2 and 4 (t2, t4) enter the
        // delay lines after the levels below have read them
        float f1[8], t2 = 0.0f, t4 = 0.0f;
        auto level1 = [&]() {
            float u, v, fs[8];
            collide_populations<GEN>(moments(f1), hx[0], hy[0], c, u, v, fs);
            float* d = rt + (i & D) * R;
            d[0 * PL] = fs[0];
            d[1 * PL] = fs[2];
            d[2 * PL] = fs[4];
            d[3 * PL] = fs[5];
            d[4 * PL] = fs[6];
            d[5 * PL] = fs[7];
            t2 = fs[1];
            t4 = fs[3];
        };
        if (l1) {
            if constexpr (CIRC) {
                // row i + 2 into the buffer row i - 2 left; row i stays in
                // buffer K until step 1 collides it below
                if (FULL || i + 2 < n1) load1((K + 2) & 3);
            } else {
                constexpr int bq = PA2 ? b : 0;
                pull_decode<S>(a, q[bq], f1, c.theta);
                // L1FIRST: collide row i before reloading its buffers (ring slot i
                // mod 4 is not among the slots the levels below read)
                if constexpr (L1FIRST) level1();
                if (FULL || i + (PA2 ? 2 : 1) < n1) load1(bq);
            }
            if (FULL || i + (LA2 ? 2 : 1) < n1) load_force(b);
        }
        // Levels T..2: local row j = i - 2(tau - 1), pulled from ring tau - 1.
#pragma unroll
        for (int tau = T; tau >= 2; --tau) {
            // active rows y0 - (T - tau) .. y0 + rows - 1 + (T - tau)
            if (!FULL && (i < 3 * (tau - 1) || i > rows + 2 * T + tau - 4)) continue;
            const int j = i - 2 * (tau - 1);
            const float* sp = rt + (tau - 2) * RP;
            const int rm = ((j - 1) & D) * R, r0 = (j & D) * R, rp = ((j + 1) & D) * R;
            float f[8];
            f[0] = sp[0 * PL + r0 - 1];          // f_p(x) = f*_p(x - c_p)
            f[1] = CIRC ? v2[tau - 2][(K + 1) & 3] : v2[tau - 2][2];   // made 3 iterations ago
            f[2] = sp[1 * PL + r0 + 1];
            f[3] = v4[tau - 2];
            f[4] = sp[2 * PL + rm - 1];
            f[5] = sp[3 * PL + rm + 1];
            f[6] = sp[4 * PL + rp + 1];
            f[7] = sp[5 * PL + rp - 1];
            const float gx = hx[2 * (tau - 1)], gy = hy[2 * (tau - 1)];
            const Mom<float> m = moments(f);
            if (tau < T) {
                float u, v, fs[8];
                collide_populations<GEN>(m, gx, gy, c, u, v, fs);
                float* d = rt + (tau - 1) * RP + r0;
                d[0 * PL] = fs[0];
                d[1 * PL] = fs[2];
                d[2 * PL] = fs[4];
                d[3 * PL] = fs[5];
                d[4 * PL] = fs[6];
                d[5 * PL] = fs[7];
                if constexpr (CIRC) {
                    v2[tau - 1][K] = fs[1];
                } else {
                    v2[tau - 1][2] = v2[tau - 1][1];
                    v2[tau - 1][1] = v2[tau - 1][0];
                    v2[tau - 1][0] = fs[1];
                }
                v4[tau - 1] = fs[3];
            } else {
                // every thread collides; only the stores are predicated
                float u, v, fs[8], c10, c01;
                post_state<S, GEN>(m, gx, gy, c, u, v, fs, c10, c01);
                if (store_ok) {
                    const I idx = (I)(ybeg + j) * nx + xs;   // row in [y0, y0 + rows), xs < nx
                    if (CHECK) {
                        check_node<S>(a, n, (int64_t)idx, acc, so, f, gx, gy, u, v);
                        if (FULL || i + 1 < iters) snap_next(i + 1);
                    }
                    store_state<S>(a, (int64_t)idx, fs, c10, c01);
                }
            }
        }
        if (l1) {
            if constexpr (CIRC) {
                pull_decode<S>(a, q[K], f1, c.theta);
                level1();
                v2[0][K] = t2;
            } else {
                if constexpr (!L1FIRST) level1();
                v2[0][2] = v2[0][1];
                v2[0][1] = v2[0][0];
                v2[0][0] = t2;
            }
            v4[0] = t4;
        }
        __syncthreads();
    };

    load1(0);
    if (PA2 && n1 > 1) load1(1);
    load_force(0);
    if (LA2 && n1 > 1) load_force(1);
    const int fb = 3 * (T - 1);                   // first iteration with every level active
    // last one whose level 1 still loads ahead
    const int fe = n1 - 1 - (LA2 || PA2 ? 2 : 1);
    if (CHECK && store_ok) snap_next(fb);         // level T's first row is y0
    const int m0 = (fb + 3) >> 2, m1 = (fe + 1) >> 2;   // groups i = 4m .. 4m + 3 within [fb, fe]
    using B0 = std::integral_constant<int, 0>;
    using B1 = std::integral_constant<int, 1>;
    using B2 = std::integral_constant<int, CIRC ? 2 : 0>;
    using B3 = std::integral_constant<int, CIRC ? 3 : 1>;
    auto iter_any = [&](int i) {
        if constexpr (CIRC) {
            switch (i & 3) {
                case 0: iter(i, std::false_type{}, B0{}); break;
                case 1: iter(i, std::false_type{}, B1{}); break;
                case 2: iter(i, std::false_type{}, B2{}); break;
                default: iter(i, std::false_type{}, B3{}); break;
            }
        } else {
            if (LA2 && (i & 1)) iter(i, std::false_type{}, B1{});
            else iter(i, std::false_type{}, B0{});
        }
    };
    int i = 0;
    if (m1 > m0) {
        for (; i < 4 * m0; ++i) iter_any(i);
        for (int m = m0; m < m1; ++m) {
            const int ib = m << 2;
            iter(ib, std::true_type{}, B0{});
            iter(ib + 1, std::true_type{}, B1{});
            iter(ib + 2, std::true_type{}, B2{});
            iter(ib + 3, std::true_type{}, B3{});
        }
        i = 4 * m1;
    }
    for (; i < iters; ++i) iter_any(i);
}

template <int S, bool GEN, int T, bool CHECK, typename I>
__global__ void __launch_bounds__(kWvW, (wv_minb<S, T>()))
k_wave(const StepParams a, const Coef<float> c, int seg) {
    extern __shared__ float wv_ring[];            // (T-1) rings of 6 planes x kWvD rows x kWvRow, staging
    const int nstrips = (a.nx + wv_ox<T>() - 1) / wv_ox<T>();
    const int strip = (int)(blockIdx.x % (unsigned)nstrips);
    const int y0 = (int)(blockIdx.x / (unsigned)nstrips) * seg;
    ResAcc<S> acc;
    wave_block<S, GEN, T, CHECK, I, true>(a, c, wv_ring, strip, y0, min(seg, a.ny - y0), acc);
    if (CHECK) residual_reduce<S>(a, acc);
}

// Destinations of the five solution fields u_x, u_y, sigma_xx, sigma_yy,
// sigma_xy (nx*ny doubles each; a null entry is not written).  Device memory,
// or pinned host memory the device can address (the recovery then writes the
// caller's arrays over the host link directly).
// tr: the lattice is the transpose of the caller's (x and y exchanged), so
// node (x, y) goes to entry x * ny + y of each destination.
struct FieldOut {
    double* p[5];
    int tr;
};

inline FieldOut field_planes(double* out, int64_t n) {
    FieldOut o;
    for (int k = 0; k < 5; ++k) o.p[k] = out + k * n;
    o.tr = 0;
    return o;
}

// Solution fields of the current state (Table 2, Eq. compute_bared), FP64.
template <int S>
__global__ void __launch_bounds__(kThreads)
k_fields(const StepParams a, const Coef<double> c, typename StoreT<S>::T theta, const FieldOut out) {
    using T = typename StoreT<S>::T;
    using G = typename StoreT<S>::G;
    const int nx = a.nx, ny = a.ny;
    const int y = blockIdx.y * BY + threadIdx.y;
    const int x = blockIdx.x * 32 + threadIdx.x;
    if (y >= ny || x >= nx) return;
    const int ym = wrap_dec(y, ny), yp = wrap_inc(y, ny);
    const int64_t r0 = (int64_t)y * nx, rm = (int64_t)ym * nx, rp = (int64_t)yp * nx;
    T f[8];
    gather<S>(a, r0, rm, rp, x, wrap_dec(x, nx), wrap_inc(x, nx), f, theta);
    const int64_t idx = r0 + x;
    const G gxs = static_cast<const G*>(a.gx)[idx], gys = static_cast<const G*>(a.gy)[idx];
    double u, v, m11, ms, md;
    if constexpr (S == S_F64) {
        const Mom<double> m = moments(f);
        u = m.m10 + 0.5 * gxs;
        v = m.m01 + 0.5 * gys;
        m11 = m.m11;
        ms = m.ms;
        md = m.md;
    } else {
        // FP32 populations: the moments as exact FP32 pairs (TwoSum), each
        // joined in FP64 once -- GB300 issues FP64 at a small fraction of the
        // FP32 rate, and this keeps the recovery's FP64 work to the joins and
        // the products of Eq. compute_bared
        const float4 w = exact_displacement(f, gxs, gys);
        u = (double)w.x + (double)w.y;
        v = (double)w.z + (double)w.w;
        float ep, eq, e13, e24, e11, e22, ed, et, es;
        const float p = two_sum(f[4], f[6], ep), q = two_sum(f[5], f[7], eq);
        const float h11 = two_sum(p, -q, e11), h22 = two_sum(p, q, e22);
        const float s13 = two_sum(f[0], f[2], e13), s24 = two_sum(f[1], f[3], e24);
        const float hd = two_sum(s13, -s24, ed), ht = two_sum(s13, s24, et);
        const float l22 = __fadd_rn(e22, __fadd_rn(ep, eq));
        const float hs = two_sum(ht, 2.0f * h22, es);   // m_s = (f1+f3) + (f2+f4) + 2 m_22
        m11 = (double)h11 + (double)__fadd_rn(e11, __fsub_rn(ep, eq));
        md = (double)hd + (double)__fadd_rn(ed, __fsub_rn(e13, e24));
        ms = (double)hs + (double)__fadd_rn(__fadd_rn(es, __fadd_rn(et, __fadd_rn(e13, e24))), 2.0f * l22);
    }
    // (FP16S: back from the state's scaled units, a power of two)
    const double un = S == S_F16S ? (double)a.hinv : 1.0;
    const double mb11 = c.b11 * m11, mbs = c.bs * ms, mbd = c.bd * md;
    const int64_t o = out.tr ? (int64_t)x * ny + y : idx;
    if (out.p[0]) out.p[0][o] = u * un;
    if (out.p[1]) out.p[1][o] = v * un;
    if (out.p[2]) out.p[2][o] = -0.5 * (mbs + mbd) * un;
    if (out.p[3]) out.p[3][o] = -0.5 * (mbs - mbd) * un;
    if (out.p[4]) out.p[4][o] = -mb11 * un;
}

// Pre-collision populations of the current state into 8 FP64 planes.
template <int S>
__global__ void __launch_bounds__(kThreads)
k_export(const StepParams a, typename StoreT<S>::T theta, double* out) {
    using T = typename StoreT<S>::T;
    const int nx = a.nx, ny = a.ny;
    const int y = blockIdx.y * BY + threadIdx.y;
    const int x = blockIdx.x * 32 + threadIdx.x;
    if (y >= ny || x >= nx) return;
    const int ym = wrap_dec(y, ny), yp = wrap_inc(y, ny);
    const int64_t r0 = (int64_t)y * nx, rm = (int64_t)ym * nx, rp = (int64_t)yp * nx;
    T f[8];
    gather<S>(a, r0, rm, rp, x, wrap_dec(x, nx), wrap_inc(x, nx), f, theta);
    const int64_t idx = r0 + x, n = (int64_t)nx * ny;
    // (FP16S: back from the state's scaled units; a power of two, exact)
    const double unscale = S == S_F16S ? (double)a.hinv : 1.0;
#pragma unroll
    for (int p = 0; p < 8; ++p) out[p * n + idx] = double(f[p]) * unscale;
}

// Load pre-collision populations f (8 FP64 planes): the stored post-collision
// value at x is f*_p(x) = f_p(x + c_p) (inverse of the pull gather).
template <int S>
__global__ void __launch_bounds__(kThreads)
k_import(const StepParams a, typename StoreT<S>::T theta, const double* in) {
    using T = typename StoreT<S>::T;
    using P = typename StoreT<S>::P;
    const int nx = a.nx, ny = a.ny;
    const int y = blockIdx.y * BY + threadIdx.y;
    const int x = blockIdx.x * 32 + threadIdx.x;
    if (y >= ny || x >= nx) return;
    const int xm = wrap_dec(x, nx), xp = wrap_inc(x, nx);
    const int ym = wrap_dec(y, ny), yp = wrap_inc(y, ny);
    const int64_t n = (int64_t)nx * ny;
    const int64_t r0 = (int64_t)y * nx, rm = (int64_t)ym * nx, rp = (int64_t)yp * nx;
    // f*_p(x) = f_p(x + c_p); FP16S: in the state's scaled units (the power
    // of two commutes with the rounding to FP32)
    const T sc = S == S_F16S ? T(a.hscale) : T(1);
    T fs[8];
    fs[0] = T(in[0 * n + r0 + xp]) * sc;
    fs[1] = T(in[1 * n + rp + x]) * sc;
    fs[2] = T(in[2 * n + r0 + xm]) * sc;
    fs[3] = T(in[3 * n + rm + x]) * sc;
    fs[4] = T(in[4 * n + rp + xp]) * sc;
    fs[5] = T(in[5 * n + rp + xm]) * sc;
    fs[6] = T(in[6 * n + rm + xm]) * sc;
    fs[7] = T(in[7 * n + rm + xp]) * sc;
    const int64_t idx = r0 + x;
    P* d = static_cast<P*>(a.dst);
    if constexpr (S == S_F16S) {
        const Mom<T> s = moments(fs);
        T nf[8];
        populations(deviation_moments(quarter(s), T(0.25) * theta), nf);
        (void)d;
        store_f16s(a, idx, nf, s.m10, s.m01);
    } else {
        (void)theta;
        for (int p = 0; p < 8; ++p) d[p * a.plane + idx] = P(fs[p]);
    }
}

// Force upload in one pass over the FP64 input (device memory, or pinned host
// memory the device can address): the force in the storage force type G, its
// max |g| over both components (non-negative doubles order like their bit
// patterns, so an unsigned 64-bit atomicMax suffices) and `bad` set by a
// non-finite entry.
template <typename G>
__global__ void k_force_ingest(const double* gx, const double* gy, G* ox, G* oy, int64_t n,
                               unsigned long long* absmax, unsigned int* bad) {
    double m = 0.0;
    unsigned int b = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double u = gx[i], v = gy[i];
        ox[i] = G(u);
        oy[i] = G(v);
        if (!(isfinite(u) && isfinite(v))) b = 1;
        m = fmax(m, fmax(fabs(u), fabs(v)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        b |= __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(absmax, (unsigned long long)__double_as_longlong(m));
        if (b) atomicOr(bad, 1u);
    }
}

// F16S: multiply every stored deviation by `factor` (a power of two).
__global__ void k_rescale_half(__half* h, int64_t count, float factor);
// Multiply `count` floats by `factor` (a power of two: exact unless the result
// leaves FP32's normal range).
__global__ void k_scale_float(float* v, int64_t count, float factor);

// Grid-level pass of the residual when the check launch wrote per-block
// partials only (StepParams::counter == nullptr): one block combines the
// nblocks partial sets (FP64) into result.
__global__ void k_residual_finish(const double* partials, int64_t nblocks, double* result);
constexpr int kFinishThreads = 1024;

// Higher-order force correction with periodic central differences (FP64).
__global__ void k_force_correct(const double* gx, const double* gy, double* ox, double* oy, int nx,
                                int ny, double d1, double d2, double d3);

// Launchers (defined per storage type).
template <int S>
struct Ops {
    using T = typename StoreT<S>::T;
    // check_blocks: grid cap of the CHECK launch (<= partials slots); one
    // block per tile below it
    static cudaError_t step(const StepParams& a, const Coef<T>& c, int V, bool gen, bool check,
                            int check_blocks, cudaStream_t st);
    static cudaError_t fields(const StepParams& a, const Coef<double>& c, T theta, const FieldOut& out,
                              cudaStream_t st);
    static cudaError_t export_pop(const StepParams& a, T theta, double* out, cudaStream_t st);
    static cudaError_t import_pop(const StepParams& a, T theta, const double* in, cudaStream_t st);
};

// FP16-shifted storage scale: stored deviation = deviation * 2^e.  At steady
// state the deviations are second moments ~ tau * grad u ~ |g| * L / (2 pi);
// e maps max|g| * max(nx, ny) to 2^8, leaving 2^7 of headroom below FP16's
// maximum and keeping values far above its smallest normal.
inline int f16s_exponent(double gmax, int nx, int ny) {
    if (!(gmax > 0.0)) return 0;
    const double L = double(nx > ny ? nx : ny);
    int e = 8 - (int)ceil(log2(gmax * L));
    return e < -60 ? -60 : (e > 60 ? 60 : e);
}

// Residual windows per check interval k: rounding keeps a converged stored
// state jittering by about J |u|, which floors a w-step residual near J / w.
// Measured (max|u^t - u^(t-w)| / max|u| long after convergence): FP64 ~3e-15;
// FP32 1.3e-7 .. 4.3e-7 on every shape and nu tried; FP16-shifted storage
// 2.5e-7 .. 1e-5, larger for a shorter lattice side (its stored deviations are
// of size ~ |grad u| ~ u / min(nx, ny)) and for larger nu.  A solve asking for
// tol starts with windows of min(64, max(1, ceil(2 J / (tol k)))) intervals of
// k steps, J = 4e-7 (FP32) or 6e-4 / min(nx, ny) (FP16S), and adapt_period
// stretches them while the residual stagnates, so a floor above the estimate
// cannot stall the solve.  The cap keeps divergence detection (made at
// checks) within 64 intervals; a tol that would need more is below what the
// storage type can resolve.
inline int check_period(int dtype, double tol, int k, int nmin) {
    const double J = dtype == S_F16S ? 6e-4 / (double)(nmin > 1 ? nmin : 1)
                                     : (dtype == S_F32 ? 4e-7 : 3e-15);
    if (!(tol > 0.0) || k < 1) return 64;
    const double p = ceil(2.0 * J / (tol * (double)k));
    return p < 1.0 ? 1 : (p > 64.0 ? 64 : (int)p);
}

// The next window length (in intervals of k steps) after a check above tol:
// doubled (up to 64) when the residual r did not fall below 0.95 of the
// previous check's r_prev.  Decay faster than 5 % per window keeps the window;
// a residual held up by the rounding floor J / w, or decaying very slowly, gets
// longer windows (which lower the floor and cost fewer checks; the stopping
// step moves by at most one window).
inline int adapt_period(int period, double r, double r_prev) {
    return (r > 0.95 * r_prev && period < 64) ? (period * 2 > 64 ? 64 : period * 2) : period;
}

inline int64_t step_tiles(int nx, int ny, int V) {
    return (int64_t)((nx + 32 * V - 1) / (32 * V)) * ((ny + BY - 1) / BY);
}

// Grid cap of the residual-check launches: one FP64 partial set per block.
constexpr int64_t kMaxCheckBlocks = int64_t(1) << 19;

// Two-step launches of a single lattice: from one full slot array up (smaller
// lattices would mostly compute duplicate slots).
inline bool step2_fits(int nx, int ny) { return nx >= kT2W && ny >= kT2H; }

inline int64_t step2_tiles(int nx, int ny) {
    return (int64_t)((nx + kT2OX - 1) / kT2OX) * ((ny + kT2OY - 1) / kT2OY);
}

// Three-step launches of a single lattice: from one full slot array up.
inline bool step3_fits(int nx, int ny) { return nx >= kT3W && ny >= kT3H; }

inline int64_t step3_tiles(int nx, int ny) {
    return (int64_t)((nx + kT3OX - 1) / kT3OX) * ((ny + kT3OY - 1) / kT3OY);
}

// Wavefront launches (k_wave) of a single lattice: from one strip width by 8
// rows up (the slot wrap is a single conditional subtraction there).
inline bool wave_fits(int nx, int ny) { return nx >= kWvW && ny >= 8; }

template <int T>
inline int64_t wave_blocks(int nx, int ny, int seg) {
    return (int64_t)((nx + wv_ox<T>() - 1) / wv_ox<T>()) * ((ny + seg - 1) / seg);
}

// T fused steps on the wavefront schedule (T = 3 or 4; check: T = 4 with the
// residual on the last step); defined with each storage type's kernels.
cudaError_t wave_f32(const StepParams& a, const Coef<float>& c, bool gen, int T, bool check, int seg,
                     cudaStream_t st);
cudaError_t wave_f16s(const StepParams& a, const Coef<float>& c, bool gen, int T, bool check, int seg,
                      cudaStream_t st);

// Three fused steps (k_step3); defined with each storage type's kernels.
cudaError_t step3_f32(const StepParams& a, const Coef<float>& c, bool gen, bool check,
                      int check_blocks, cudaStream_t st);
cudaError_t step3_f16s(const StepParams& a, const Coef<float>& c, bool gen, bool check,
                       int check_blocks, cudaStream_t st);

// Two fused steps (k_step2) of FP32 or FP16-shifted storage; defined with
// each storage type's kernels.
cudaError_t step2_f32(const StepParams& a, const Coef<float>& c, bool gen, bool check,
                      int check_blocks, cudaStream_t st);
cudaError_t step2_f16s(const StepParams& a, const Coef<float>& c, bool gen, bool check,
                       int check_blocks, cudaStream_t st);

inline dim3 step_grid(int nx, int ny, int V) {
    return dim3((unsigned)((nx + 32 * V - 1) / (32 * V)), (unsigned)((ny + BY - 1) / BY));
}

}  // namespace lbm
