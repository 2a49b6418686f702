// lbm_core.cuh -- per-node arithmetic of the periodic lattice Boltzmann scheme
// for linear elasticity (Boolakee, Geier, De Lorenzis, arXiv 2208.14870),
// shared by every kernel of the library.
//
// Populations are kept in the paper's one-index order (Sec. 4, population
// table): c_1..c_8 = (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1),
// stored here as f[0..7].  Moments use the paper's moment order
// 10, 01, 11, s, d, 12, 21, 22 (Sec. 4, moment table).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Rounding is spelled out wherever it could depend on the compiler: a
// product that is not exact is either rounded on its own (rmul, never fused
// into a later add) or fused on purpose (fmad).  Products with 1/2, 1/4 and 2
// are exact, so fusing them or not gives the same bits.  Every kernel that
// runs this arithmetic (one step per launch, two steps per launch, the
// batched arena) therefore computes the same bits for the same inputs.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return fma(a, b, c); }

// Moments of the collision basis.
template <typename T>
struct Mom {
    T m10, m01, m11, ms, md, m12, m21, m22;
};

// Per-lattice constants of the collision in compute precision, in the
// quarter form collide returns (every factor of a second-order moment
// divided by 4; see collide):
//   q11 = (1 - w11)/4, qs = (1 - ws)/4, qd = (1 - wd)/4     (Eq. collision, m^eq = 0)
//   qw12t = w12 theta / 4, q12 = (1 - w12)/4, ...          (m^eq_12 = theta mbar_10)
//   qtheta = theta / 4; theta itself for the FP16-shifted store
template <typename T>
struct Coef {
    T q11, qs, qd;
    T qw12t, q12, qw21t, q21, q22;
    T qtheta, theta;
    T b11, bs, bd;   // 1 - w/2 (bared moments, Eq. compute_bared)
};

// Raw moments of eight populations, Eq. moments and Eq. replace_raw, written
// as a butterfly: with p = f5 + f7, q = f6 + f8, r = f5 - f7, s = f6 - f8,
//   m11 = p - q, m22 = p + q, m12 = r - s, m21 = r + s,
//   m10 = (f1 - f3) + m12, m01 = (f2 - f4) + m21,
//   ms = (f1 + f3) + (f2 + f4) + 2 m22, md = (f1 + f3) - (f2 + f4).
template <typename T>
__device__ __forceinline__ Mom<T> moments(const T f[8]) {
    Mom<T> m;
    const T p = f[4] + f[6], q = f[5] + f[7];
    const T r = f[4] - f[6], s = f[5] - f[7];
    m.m11 = p - q;
    m.m22 = p + q;
    m.m12 = r - s;
    m.m21 = r + s;
    m.m10 = (f[0] - f[2]) + m.m12;
    m.m01 = (f[1] - f[3]) + m.m21;
    const T s13 = f[0] + f[2], s24 = f[1] + f[3];
    m.ms = (s13 + s24) + T(2) * m.m22;
    m.md = s13 - s24;
    return m;
}

// Collision in moment space (Algorithm 1, collision block):
//   mbar_10 = m_10 + g_x/2, mbar_01 = m_01 + g_y/2          (Eqs. coll10, coll01)
//   m*_a = w_a m^eq_a + (1 - w_a) m_a, Table 1 equilibria  (Eq. collision)
//   m*_10 = mbar_10 + g_x/2, m*_01 = mbar_01 + g_y/2       (Eqs. coll10post, coll01post)
// GEN = false is the standard case w_12 = w_21 = w_22 = 1 (Sec. 3.3.2),
// where m*_12 = theta u, m*_21 = theta v, m*_22 = 0.
// u, v receive the displacement mbar_10, mbar_01 (Table 2).
//
// Returned in the form the back-transform consumes ("quarter form"): m*_10
// and m*_01 as they are, the moments of order two and higher (11, s, d, 12,
// 21, 22) divided by 4.  The 1/4 rides on the coefficients (Coef), and since
// 4 is a power of two, (c/4) * m rounds to exactly (c * m)/4: the stored
// populations are the same bits as without it, at six fewer multiplications
// per node.
// The displacement u = mbar_10, v = mbar_01 of raw moments m (Eqs. coll10,
// coll01; Table 2).
template <typename T>
__device__ __forceinline__ void displacement(const Mom<T>& m, T gx, T gy, T& u, T& v) {
    u = m.m10 + T(0.5) * gx;
    v = m.m01 + T(0.5) * gy;
}

template <typename T, bool GEN>
__device__ __forceinline__ Mom<T> collide(const Mom<T>& m, T gx, T gy, const Coef<T>& c,
                                          T& u, T& v) {
    Mom<T> s;
    displacement(m, gx, gy, u, v);
    s.m10 = m.m10 + gx;
    s.m01 = m.m01 + gy;
    s.m11 = rmul(c.q11, m.m11);
    s.ms = rmul(c.qs, m.ms);
    s.md = rmul(c.qd, m.md);
    if (GEN) {
        s.m12 = fmad(c.qw12t, u, rmul(c.q12, m.m12));
        s.m21 = fmad(c.qw21t, v, rmul(c.q21, m.m21));
        s.m22 = rmul(c.q22, m.m22);
    } else {
        s.m12 = rmul(c.qtheta, u);
        s.m21 = rmul(c.qtheta, v);
        s.m22 = T(0);
    }
    return s;
}

// Raw moments in quarter form (for states that did not come from collide).
template <typename T>
__device__ __forceinline__ Mom<T> quarter(Mom<T> m) {
    const T q = T(0.25);
    m.m11 = q * m.m11;
    m.ms = q * m.ms;
    m.md = q * m.md;
    m.m12 = q * m.m12;
    m.m21 = q * m.m21;
    m.m22 = q * m.m22;
    return m;
}

// Back-transformation f = M^-1 m (Eq. moments_post solved in closed form),
// from the quarter form (m11 ... m22 below are the moments divided by 4):
//   A = m10 - 4 m12, B = m01 - 4 m21, P = ms - 2 m22 + md, Q = ms - 2 m22 - md
//   f1 = P + A/2, f3 = P - A/2, f2 = Q + B/2, f4 = Q - B/2
//   f5 = m22 + m11 + m12 + m21, f6 = m22 - m11 - m12 + m21,
//   f7 = m22 + m11 - m12 - m21, f8 = m22 - m11 + m12 - m21.
// ZERO22: the standard rates (w_22 = 1, so m*_22 = m^eq_22 = 0) drop m22
// from the sums; that changes at most the sign of a zero population, so every
// kernel running the standard rates uses this form.
template <bool ZERO22 = false, typename T>
__device__ __forceinline__ void populations(const Mom<T>& s, T f[8]) {
    const T A = fmad(T(-4), s.m12, s.m10), B = fmad(T(-4), s.m21, s.m01);
    if (ZERO22) {
        const T P = s.ms + s.md, Q = s.ms - s.md;
        f[0] = fmad(T(0.5), A, P);
        f[2] = fmad(T(-0.5), A, P);
        f[1] = fmad(T(0.5), B, Q);
        f[3] = fmad(T(-0.5), B, Q);
        const T h3 = s.m12 + s.m21, h4 = s.m21 - s.m12;
        f[4] = s.m11 + h3;
        f[6] = s.m11 - h3;
        f[5] = h4 - s.m11;
        f[7] = -s.m11 - h4;
        return;
    }
    const T t = fmad(T(-2), s.m22, s.ms);
    const T P = t + s.md, Q = t - s.md;
    f[0] = fmad(T(0.5), A, P);
    f[2] = fmad(T(-0.5), A, P);
    f[1] = fmad(T(0.5), B, Q);
    f[3] = fmad(T(-0.5), B, Q);
    const T h1 = s.m22 + s.m11, h2 = s.m22 - s.m11;
    const T h3 = s.m12 + s.m21, h4 = s.m21 - s.m12;
    f[4] = h1 + h3;
    f[6] = h1 - h3;
    f[5] = h2 + h4;
    f[7] = h2 - h4;
}

// Post-collision populations straight from the raw moments: collide, then
// populations (the standard rates drop m*_22).  (Merging the two into fused
// multiply-adds on the raw moments saves two operations per node but measured
// slower in the four-step wavefront kernel.)
template <bool GEN, typename T>
__device__ __forceinline__ void collide_populations(const Mom<T>& m, T gx, T gy, const Coef<T>& c, T& u, T& v,
                                                    T f[8]) {
    populations<!GEN>(collide<T, GEN>(m, gx, gy, c, u, v), f);
}

// Shifted FP16 storage.  The equilibrium-type part of a post-collision state
// with first moments (c10, c01) is E = M^-1 (c10, c01, 0, 0, 0, theta c10,
// theta c01, 0):
//   E1 = k1 c10, E3 = -k1 c10, E2 = k1 c01, E4 = -k1 c01   (k1 = (1 - theta)/2)
//   E5 = k5 (c10 + c01), E6 = k5 (c01 - c10), E7 = -k5 (c10 + c01),
//   E8 = k5 (c10 - c01)                                     (k5 = theta/4)
// The stored deviation is N = f* - E = M^-1 (0, 0, m*_11, m*_s, m*_d,
// m*_12 - theta m*_10, m*_21 - theta m*_01, m*_22), which is O(eps) of f*.
// (Quarter form in and out: the m*_12 - theta m*_10 terms are divided by 4;
// qtheta = theta / 4.)
template <typename T>
__device__ __forceinline__ Mom<T> deviation_moments(const Mom<T>& s, T qtheta) {
    Mom<T> n = s;
    n.m10 = T(0);
    n.m01 = T(0);
    n.m12 = fmad(-qtheta, s.m10, s.m12);
    n.m21 = fmad(-qtheta, s.m01, s.m21);
    return n;
}

// Error-free FP32 transformations for the steady-state residual.  GB300's
// FP64 pipe issues about 1/64 of the FP32 rate, so the residual of FP32 and
// FP16-shifted storage evaluates the displacement in FP32 pairs (hi + lo)
// instead of FP64 per node: two_sum is Knuth's TwoSum (s + e == a + b
// exactly, six FP32 additions, no branch), fast_two_sum Dekker's form for
// |a| >= |b| (three additions).  Every operation is written with explicit
// rounding so that no compiler contraction or reassociation can touch it.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

__device__ __forceinline__ float fast_two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
    return s;
}

// The displacement of eight FP32 pre-collision populations, u = mbar_10 =
// m_10 + g_x / 2 and v = mbar_01 (Eqs. coll10, coll01; Table 2), as FP32
// pairs (u_hi, u_lo, v_hi, v_lo).  The sums are the moment butterfly's
// (moments(), then collide's half force), so u_hi + u_lo carries exactly the
// value the butterfly rounds, with each addition's rounding error recovered
// by two_sum: m_12 = r - s with r = f5 - f7, s = f6 - f8, m_10 = (f1 - f3) +
// m_12, u = m_10 + g_x / 2 (and m_21 = r + s, m_01 = (f2 - f4) + m_21).  The
// error terms are summed in FP32, so the pair is exact to about 2^-44 of the
// largest partial sum; the hi parts are the FP32 values the collision uses.
__device__ __forceinline__ float4 exact_displacement(const float f[8], float gx, float gy) {
    float er, es, e12, e21, ea, eb, e10, e01, eu, ev;
    const float r = two_sum(f[4], -f[6], er);
    const float s = two_sum(f[5], -f[7], es);
    const float m12 = two_sum(r, -s, e12);
    const float m21 = two_sum(r, s, e21);
    const float a = two_sum(f[0], -f[2], ea);
    const float b = two_sum(f[1], -f[3], eb);
    const float m10 = two_sum(a, m12, e10);
    const float m01 = two_sum(b, m21, e01);
    const float u = two_sum(m10, 0.5f * gx, eu);
    const float v = two_sum(m01, 0.5f * gy, ev);
    const float ulo = __fadd_rn(__fadd_rn(__fadd_rn(eu, e10), __fadd_rn(ea, e12)), __fsub_rn(er, es));
    const float vlo = __fadd_rn(__fadd_rn(__fadd_rn(ev, e01), __fadd_rn(eb, e21)), __fadd_rn(er, es));
    float4 d;
    d.x = two_sum(u, ulo, d.y);
    d.z = two_sum(v, vlo, d.w);
    return d;
}

__device__ __forceinline__ int wrap_dec(int i, int n) { return i == 0 ? n - 1 : i - 1; }
__device__ __forceinline__ int wrap_inc(int i, int n) { return i + 1 == n ? 0 : i + 1; }

}  // namespace lbm
