/*
 * lbm_oracle.c -- plain, slow FP64 CPU restatement of the lattice Boltzmann
 * scheme for quasi-static linear elasticity of Boolakee, Geier and De Lorenzis
 * (arXiv 2208.14870), "A new lattice Boltzmann scheme for linear elastic
 * solids: periodic problems".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA library is
 * checked against.  Only tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * One pseudo-time step is the composition of the paper's defining equations,
 * applied node by node and then as a shift of every population plane:
 *   f(t+1) = S (M^-1 C(M f(t), g)),
 * with M the raw-moment map of Eq. moments (rewritten by Eq. replace_raw), C
 * the collision of Eq. collision with the Table 1 equilibria and the force
 * split symmetrically around it (Eqs. coll10, coll01, coll10post,
 * coll01post), M^-1 the solution of Eq. moments_post, and S the streaming of
 * Eq. streaming with the periodic wrap of Sec. 5.1.  The pieces:
 *   - populations f_ij, i,j in {-1,0,1}; the D2Q8 set drops the rest
 *     population f_00 (Sec. 3.3.2, remark on m_00); an optional ninth slot
 *     carries f_00 to show that it is inert;
 *   - raw countable moments m_ab = sum_ij i^a j^b f_ij (Eq. moments);
 *   - spherical / deviatoric split m_s = m_20 + m_02, m_d = m_20 - m_02
 *     (Eq. replace_raw);
 *   - half forcing before collision, bared first moments
 *     mbar_10 = m_10 + g_x/2 (Eqs. coll10, coll01);
 *   - equilibria of Table 1: m_11^eq = m_s^eq = m_d^eq = m_22^eq = 0,
 *     m_12^eq = theta*mbar_10, m_21^eq = theta*mbar_01;
 *   - relaxation m*_a = w_a m^eq_a + (1 - w_a) m_a (Eq. collision) for
 *     a in {11, s, d, 12, 21, 22}; m_00 is not collided;
 *   - half forcing after collision m*_10 = mbar_10 + g_x/2 (Eqs. coll10post,
 *     coll01post);
 *   - back-transformation: m*_20, m*_02 from m*_s, m*_d (inverse of
 *     Eq. replace_raw), then the linear system m*_ab = sum_ij i^a j^b f*_ij
 *     (Eq. moments_post) is solved for f*_ij.  The system matrix is built
 *     from the velocity table and inverted once by Gauss-Jordan elimination;
 *   - streaming f_ij(x + c_ij, t + 1) = f*_ij(x, t) (Eq. streaming) with the
 *     periodic wrap of Sec. 5.1 (outgoing populations re-enter on the
 *     opposite side).
 *
 * Solution fields (Table 2 and Eq. compute_bared), in lattice units:
 *   u_x = mbar_10, u_y = mbar_01 (Table 2 prints mbar_10 for u_y; the
 *   identification Eq. ident01 and the grid-norm definition in Sec. 6.1 give
 *   mbar_01, which is used here);
 *   sigma_xx = -(mbar_s + mbar_d)/2, sigma_yy = -(mbar_s - mbar_d)/2,
 *   sigma_xy = -mbar_11, with mbar_a = (w_a/2) m_a^eq + (1 - w_a/2) m_a.
 *   The paper's dimensionless stress is these values divided by
 *   epsilon = dx/L.
 *
 * Layout of every population array: q planes of nx*ny doubles, plane p holds
 * population p (order of the paper's Table "map between one-index and
 * two-index notations": 10, 01, -10, 0-1, 11, -11, -1-1, 1-1, then 00 when
 * q == 9), node (x, y) at index y*nx + x.
 *
 * Compile with -ffp-contract=off so that no fused multiply-add changes the
 * rounding of the plain expressions below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Velocity table (paper, Table "map between one-index and two-index
 * notations for the populations"), plus the rest population as index 8. */
static const int CX[9] = {1, 0, -1, 0, 1, -1, -1, 1, 0};
static const int CY[9] = {0, 1, 0, -1, 1, 1, -1, -1, 0};

/* Raw moment exponents (a, b) of the rows of the moment system, in the
 * paper's moment order 10, 01, 11, 20, 02, 12, 21, 22, then 00.  Rows 3 and
 * 4 are the raw second moments m_20 and m_02, which Eq. replace_raw turns
 * into m_s and m_d. */
static const int MA[9] = {1, 0, 1, 2, 0, 1, 2, 2, 0};
static const int MB[9] = {0, 1, 1, 0, 2, 2, 1, 2, 0};

static double ipow(int base, int e) {
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= (double)base;
    return r;
}

/* Inverse of the raw-moment matrix T[r][p] = CX[p]^a_r * CY[p]^b_r for the
 * first q velocities and moments, by Gauss-Jordan elimination with partial
 * pivoting.  Returns 0 on success. */
static int raw_moment_inverse(int q, double inv[9][9]) {
    double a[9][18];
    for (int r = 0; r < q; ++r) {
        for (int p = 0; p < q; ++p) a[r][p] = ipow(CX[p], MA[r]) * ipow(CY[p], MB[r]);
        for (int p = 0; p < q; ++p) a[r][q + p] = (r == p) ? 1.0 : 0.0;
    }
    for (int col = 0; col < q; ++col) {
        int piv = col;
        for (int r = col + 1; r < q; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (fabs(a[piv][col]) < 1e-12) return -1;
        if (piv != col)
            for (int c = 0; c < 2 * q; ++c) {
                double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t;
            }
        double d = a[col][col];
        for (int c = 0; c < 2 * q; ++c) a[col][c] /= d;
        for (int r = 0; r < q; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            if (m == 0.0) continue;
            for (int c = 0; c < 2 * q; ++c) a[r][c] -= m * a[col][c];
        }
    }
    for (int r = 0; r < q; ++r)
        for (int c = 0; c < q; ++c) inv[r][c] = a[r][q + c];
    return 0;
}

/* Relaxation rates and theta.  w[0..5] = w_11, w_s, w_d, w_12, w_21, w_22. */
typedef struct {
    double w11, ws, wd, w12, w21, w22, theta;
} rates_t;

/* Moments in the collision basis of one node: 10, 01, 11, s, d, 12, 21, 22
 * (paper's moment table), and m_00 in slot 8 when q == 9. */
static void node_moments(int q, const double *f, double m[9]) {
    double raw[9];
    for (int r = 0; r < q; ++r) {
        double s = 0.0;
        for (int p = 0; p < q; ++p) s += ipow(CX[p], MA[r]) * ipow(CY[p], MB[r]) * f[p];
        raw[r] = s;
    }
    m[0] = raw[0];                 /* m_10 */
    m[1] = raw[1];                 /* m_01 */
    m[2] = raw[2];                 /* m_11 */
    m[3] = raw[3] + raw[4];        /* m_s = m_20 + m_02 */
    m[4] = raw[3] - raw[4];        /* m_d = m_20 - m_02 */
    m[5] = raw[5];                 /* m_12 */
    m[6] = raw[6];                 /* m_21 */
    m[7] = raw[7];                 /* m_22 */
    if (q == 9) m[8] = raw[8];     /* m_00 */
}

/* The per-node map f* = M^-1 C(M f, g): raw moments of the pre-collision
 * populations, the collision of Eq. collision on the moment vector (Table 1
 * equilibria; the force enters half before and half after, Eqs. coll10 and
 * coll10post), and the post-collision populations from Eq. moments_post. */
static void collide_node(int q, const double inv[9][9], const rates_t *w,
                         const double *f, double gx, double gy, double *fs) {
    double m[9];
    node_moments(q, f, m);
    /* half forcing before collision (Eqs. coll10, coll01) */
    double mb10 = m[0] + gx / 2.0;
    double mb01 = m[1] + gy / 2.0;
    /* local equilibria (Table 1) */
    double eq11 = 0.0, eqs = 0.0, eqd = 0.0, eq22 = 0.0;
    double eq12 = w->theta * mb10;
    double eq21 = w->theta * mb01;
    /* relaxation (Eq. collision) */
    double s11 = w->w11 * eq11 + (1.0 - w->w11) * m[2];
    double ss = w->ws * eqs + (1.0 - w->ws) * m[3];
    double sd = w->wd * eqd + (1.0 - w->wd) * m[4];
    double s12 = w->w12 * eq12 + (1.0 - w->w12) * m[5];
    double s21 = w->w21 * eq21 + (1.0 - w->w21) * m[6];
    double s22 = w->w22 * eq22 + (1.0 - w->w22) * m[7];
    /* half forcing after collision (Eqs. coll10post, coll01post) */
    double s10 = mb10 + gx / 2.0;
    double s01 = mb01 + gy / 2.0;
    /* back to raw moments (inverse of Eq. replace_raw) */
    double raw[9];
    raw[0] = s10;
    raw[1] = s01;
    raw[2] = s11;
    raw[3] = (ss + sd) / 2.0;  /* m*_20 */
    raw[4] = (ss - sd) / 2.0;  /* m*_02 */
    raw[5] = s12;
    raw[6] = s21;
    raw[7] = s22;
    if (q == 9) raw[8] = m[8]; /* m_00 is not collided */
    /* solve Eq. moments_post for the post-collision populations */
    for (int p = 0; p < q; ++p) {
        double s = 0.0;
        for (int r = 0; r < q; ++r) s += inv[p][r] * raw[r];
        fs[p] = s;
    }
}

static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

/*
 * One or more pseudo-time steps f(t+1) = S(M^-1 C(M f(t), g)): the per-node
 * map at every node, then streaming (Eq. streaming).  f_in holds the
 * pre-collision populations at step t; f_out
 * receives them at step t + nsteps.  `tmp` is caller-provided scratch of the
 * same size as f_in.  f_in and f_out may be the same array.
 * Returns 0 on success, -1 on bad arguments.
 */
int oracle_run(int nx, int ny, int q, const double *f_in, const double *gx,
               const double *gy, const double *wv, long nsteps, double *f_out,
               double *tmp) {
    if (nx < 1 || ny < 1 || (q != 8 && q != 9) || nsteps < 0) return -1;
    double inv[9][9];
    if (raw_moment_inverse(q, inv) != 0) return -1;
    rates_t w = {wv[0], wv[1], wv[2], wv[3], wv[4], wv[5], wv[6]};
    const size_t n = (size_t)nx * (size_t)ny;
    if (f_out != f_in) memcpy(f_out, f_in, sizeof(double) * q * n);
    double *cur = f_out, *nxt = tmp;
    for (long t = 0; t < nsteps; ++t) {
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t idx = (size_t)y * nx + x;
                double f[9], fs[9];
                for (int p = 0; p < q; ++p) f[p] = cur[p * n + idx];
                collide_node(q, inv, &w, f, gx[idx], gy[idx], fs);
                /* streaming (Eq. streaming), periodic wrap (Sec. 5.1) */
                for (int p = 0; p < q; ++p) {
                    int xd = wrap(x + CX[p], nx), yd = wrap(y + CY[p], ny);
                    nxt[p * n + (size_t)yd * nx + xd] = fs[p];
                }
            }
        double *t2 = cur; cur = nxt; nxt = t2;
    }
    if (cur != f_out) memcpy(f_out, cur, sizeof(double) * q * n);
    return 0;
}

/*
 * Collision only (no streaming) at every node: f_star = collide(f).  Used by
 * tests that look at the collision map on its own.
 */
int oracle_collide(int nx, int ny, int q, const double *f, const double *gx,
                   const double *gy, const double *wv, double *f_star) {
    if (nx < 1 || ny < 1 || (q != 8 && q != 9)) return -1;
    double inv[9][9];
    if (raw_moment_inverse(q, inv) != 0) return -1;
    rates_t w = {wv[0], wv[1], wv[2], wv[3], wv[4], wv[5], wv[6]};
    const size_t n = (size_t)nx * (size_t)ny;
    for (size_t idx = 0; idx < n; ++idx) {
        double fl[9], fs[9];
        for (int p = 0; p < q; ++p) fl[p] = f[p * n + idx];
        collide_node(q, inv, &w, fl, gx[idx], gy[idx], fs);
        for (int p = 0; p < q; ++p) f_star[p * n + idx] = fs[p];
    }
    return 0;
}

/*
 * Moments of the pre-collision state in the collision basis, 8 (or 9)
 * planes: m_10, m_01, m_11, m_s, m_d, m_12, m_21, m_22 (, m_00).
 */
int oracle_moments(int nx, int ny, int q, const double *f, double *m_out) {
    if (nx < 1 || ny < 1 || (q != 8 && q != 9)) return -1;
    const size_t n = (size_t)nx * (size_t)ny;
    for (size_t idx = 0; idx < n; ++idx) {
        double fl[9], m[9];
        for (int p = 0; p < q; ++p) fl[p] = f[p * n + idx];
        node_moments(q, fl, m);
        for (int r = 0; r < q; ++r) m_out[r * n + idx] = m[r];
    }
    return 0;
}

/*
 * Solution fields of the pre-collision state (Table 2, Eq. compute_bared),
 * lattice units.  out: 5 planes u_x, u_y, sigma_xx, sigma_yy, sigma_xy.
 */
int oracle_fields(int nx, int ny, int q, const double *f, const double *gx,
                  const double *gy, const double *wv, double *out) {
    if (nx < 1 || ny < 1 || (q != 8 && q != 9)) return -1;
    rates_t w = {wv[0], wv[1], wv[2], wv[3], wv[4], wv[5], wv[6]};
    const size_t n = (size_t)nx * (size_t)ny;
    for (size_t idx = 0; idx < n; ++idx) {
        double fl[9], m[9];
        for (int p = 0; p < q; ++p) fl[p] = f[p * n + idx];
        node_moments(q, fl, m);
        double mb10 = m[0] + gx[idx] / 2.0;       /* Eq. coll10 */
        double mb01 = m[1] + gy[idx] / 2.0;       /* Eq. coll01 */
        /* Eq. compute_bared with the Table 1 equilibria (all zero here) */
        double mb11 = (w.w11 / 2.0) * 0.0 + (1.0 - w.w11 / 2.0) * m[2];
        double mbs = (w.ws / 2.0) * 0.0 + (1.0 - w.ws / 2.0) * m[3];
        double mbd = (w.wd / 2.0) * 0.0 + (1.0 - w.wd / 2.0) * m[4];
        out[0 * n + idx] = mb10;
        out[1 * n + idx] = mb01;
        out[2 * n + idx] = -(mbs + mbd) / 2.0;
        out[3 * n + idx] = -(mbs - mbd) / 2.0;
        out[4 * n + idx] = -mb11;
    }
    return 0;
}

/* The inverse raw-moment matrix, for tests (q x q, row-major). */
int oracle_raw_moment_inverse(int q, double *out) {
    double inv[9][9];
    if ((q != 8 && q != 9) || raw_moment_inverse(q, inv) != 0) return -1;
    for (int r = 0; r < q; ++r)
        for (int c = 0; c < q; ++c) out[r * q + c] = inv[r][c];
    return 0;
}
