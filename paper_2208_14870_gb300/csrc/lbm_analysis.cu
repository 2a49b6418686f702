// lbm_analysis.cu -- von Neumann stability of the scheme (Sec. 4): the
// spectral radius of the one-step amplification matrix L(k) = S(k) A,
// sampled over wave vectors, computed on the host.
//
// A = M^-1 Lambda M^eq + M^-1 (I - Lambda) M (Eq. lbmvector) with the Table 1
// equilibria (m_12^eq = theta m_10, m_21^eq = theta m_01) and
// S(k) = diag(exp(-i k.c_p)).  The spectral radius is obtained from
// Gelfand's formula rho(L) = lim ||L^n||^(1/n), evaluating L^(2^m) by m
// repeated squarings with renormalisation (n = 2^48), which needs no
// eigenvalue solver and is insensitive to defective eigenvalues.
#include <cmath>
#include <complex>

#include "../../include/lbm.h"

namespace {

using cd = std::complex<double>;

constexpr int kCx[8] = {1, 0, -1, 0, 1, -1, -1, 1};
constexpr int kCy[8] = {0, 1, 0, -1, 1, 1, -1, -1};

double ipow(int b, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

// Moment matrix rows 10, 01, 11, s, d, 12, 21, 22 (Eq. moments, Eq. replace_raw).
void moment_matrix(double M[8][8]) {
    for (int p = 0; p < 8; ++p) {
        const int x = kCx[p], y = kCy[p];
        M[0][p] = x;
        M[1][p] = y;
        M[2][p] = x * y;
        M[3][p] = ipow(x, 2) + ipow(y, 2);
        M[4][p] = ipow(x, 2) - ipow(y, 2);
        M[5][p] = x * ipow(y, 2);
        M[6][p] = ipow(x, 2) * y;
        M[7][p] = ipow(x, 2) * ipow(y, 2);
    }
}

bool invert(const double A[8][8], double out[8][8]) {
    double a[8][16];
    for (int r = 0; r < 8; ++r)
        for (int c = 0; c < 16; ++c) a[r][c] = c < 8 ? A[r][c] : (c - 8 == r ? 1.0 : 0.0);
    for (int col = 0; col < 8; ++col) {
        int piv = col;
        for (int r = col + 1; r < 8; ++r)
            if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
        if (std::fabs(a[piv][col]) < 1e-12) return false;
        for (int c = 0; c < 16; ++c) std::swap(a[col][c], a[piv][c]);
        const double d = a[col][col];
        for (int c = 0; c < 16; ++c) a[col][c] /= d;
        for (int r = 0; r < 8; ++r)
            if (r != col && a[r][col] != 0.0) {
                const double m = a[r][col];
                for (int c = 0; c < 16; ++c) a[r][c] -= m * a[col][c];
            }
    }
    for (int r = 0; r < 8; ++r)
        for (int c = 0; c < 8; ++c) out[r][c] = a[r][c + 8];
    return true;
}

void matmul(const cd A[8][8], const cd B[8][8], cd C[8][8]) {
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            cd s = 0.0;
            for (int k = 0; k < 8; ++k) s += A[i][k] * B[k][j];
            C[i][j] = s;
        }
}

double spectral_radius_of(cd L[8][8]) {
    double logscale = 0.0;
    cd B[8][8], T[8][8];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) B[i][j] = L[i][j];
    const int m = 48;
    for (int it = 0; it < m; ++it) {
        matmul(B, B, T);
        double nrm = 0.0;
        for (int i = 0; i < 8; ++i)
            for (int j = 0; j < 8; ++j) nrm = std::fmax(nrm, std::abs(T[i][j]));
        if (nrm == 0.0) return 0.0;
        for (int i = 0; i < 8; ++i)
            for (int j = 0; j < 8; ++j) B[i][j] = T[i][j] / nrm;
        logscale = 2.0 * logscale + std::log(nrm);
    }
    return std::exp(std::ldexp(logscale, -m));
}

}  // namespace

extern "C" int lbm_spectral_radius(double lambda, double mu, double theta, double tau12,
                                   double tau22, int nk, int nphi, double* rho) {
    if (!rho || nk < 2 || nphi < 1) return LBM_ERR_ARG;
    if (theta == 0.0) theta = 1.0 / 3.0;
    if (tau12 == 0.0) tau12 = 0.5;
    if (tau22 == 0.0) tau22 = 0.5;
    if (!(mu > 0.0) || !(lambda + mu > 0.0) || !(theta > 0.0 && theta < 1.0)) return LBM_ERR_ARG;
    const double K = lambda + mu;
    const double w[8] = {0.0,
                         0.0,
                         1.0 / (mu / theta + 0.5),
                         1.0 / (2.0 * K / (1.0 + theta) + 0.5),
                         1.0 / (2.0 * mu / (1.0 - theta) + 0.5),
                         1.0 / (tau12 + 0.5),
                         1.0 / (tau12 + 0.5),
                         1.0 / (tau22 + 0.5)};
    double M[8][8], Mi[8][8], Meq[8][8] = {};
    moment_matrix(M);
    if (!invert(M, Mi)) return LBM_ERR_ARG;
    for (int p = 0; p < 8; ++p) {
        Meq[0][p] = M[0][p];
        Meq[1][p] = M[1][p];
        Meq[5][p] = theta * M[0][p];
        Meq[6][p] = theta * M[1][p];
    }
    // A = Mi (Lambda Meq + (I - Lambda) M)
    double inner[8][8], A[8][8];
    for (int r = 0; r < 8; ++r)
        for (int p = 0; p < 8; ++p) inner[r][p] = w[r] * Meq[r][p] + (1.0 - w[r]) * M[r][p];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            double s = 0.0;
            for (int r = 0; r < 8; ++r) s += Mi[i][r] * inner[r][j];
            A[i][j] = s;
        }
    const double pi = 3.14159265358979323846;
    double best = 0.0;
    for (int a = 0; a < nphi; ++a) {
        const double phi = nphi == 1 ? 0.0 : 0.25 * pi * a / (nphi - 1);
        for (int b = 0; b < nk; ++b) {
            const double kh = pi * b / (nk - 1);
            const double k1 = kh * std::cos(phi), k2 = kh * std::sin(phi);
            cd L[8][8];
            for (int i = 0; i < 8; ++i) {
                const cd s = std::exp(cd(0.0, -(k1 * kCx[i] + k2 * kCy[i])));
                for (int j = 0; j < 8; ++j) L[i][j] = s * A[i][j];
            }
            best = std::fmax(best, spectral_radius_of(L));
        }
    }
    *rho = best;
    return LBM_OK;
}
