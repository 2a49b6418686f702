"""Pins of the error-analysis helpers of Sec. 4 / Appendices B and C.

The oracle's transcription of the printed constants is compared with the
scheme's exact discrete leading error (per-mode closed form, extrapolated in
N), which pins the parts of Appendix B that are consistent with the scheme and
documents the parts that are not (readings recorded in the design notes)."""
import numpy as np
import pytest

import oracle
import oracle.fourier as F
import workloads as W

P = pytest.importorskip("paper_2208_14870_gb300")


@pytest.mark.parametrize("E,nu", [(0.3, 0.25), (0.11, 0.8), (1.0, 0.3), (0.05, 0.6)])
@pytest.mark.parametrize("t12,t22", [(0.5, 0.5), (0.9, 0.5), (0.5, 1.5)])
def test_transverse_constant_matches_exact_discrete_error(E, nu, t12, t22):
    """C5 - mu D3 (printed) equals minus the exact transverse leading-error
    coefficient for every modulus, Poisson ratio and higher-order rate."""
    c = oracle.error_constants_printed(E, nu, tau12=t12, tau22=t22)
    lam, mu = oracle.lame_2d(E, nu)
    a1, a5 = oracle.leading_error_axis(E, nu, tau12=t12, tau22=t22)
    printed = c[4] - mu * c[7]
    assert abs(a5 + printed) < 2e-3 * abs(printed) + 1e-7


@pytest.mark.parametrize("t12,t22", [(0.5, 0.5), (0.9, 0.5), (0.5, 1.5)])
def test_longitudinal_constant_matches_at_nu_zero(t12, t22):
    """At nu = 0 the printed C1 - (mu + K) D1 equals minus the exact
    longitudinal leading-error coefficient."""
    for E in (0.1, 0.4):
        c = oracle.error_constants_printed(E, 0.0, tau12=t12, tau22=t22)
        lam, mu = oracle.lame_2d(E, 0.0)
        a1, a5 = oracle.leading_error_axis(E, 0.0, tau12=t12, tau22=t22)
        printed = c[0] - (mu + lam + mu) * c[5]
        assert abs(a1 + printed) < 2e-3 * abs(printed)


def test_longitudinal_exact_error_is_linear_in_E_unlike_printed():
    """Reading recorded in the design notes: the exact longitudinal coefficient
    is linear in E~ (its E^2 and E^3 parts vanish), whereas the printed
    C1 - (mu + K) D1 keeps an E^2 term theta (nu - theta) tau12 E^2 / ((1 - theta^2)
    (1 - nu^2)^2) (1 - 1/(1 - nu^2)) that vanishes only at nu = 0."""
    nu = 0.8
    Es = np.array([0.05, 0.1, 0.2, 0.4])
    exact = np.array([-oracle.leading_error_axis(E, nu)[0] for E in Es])
    V = np.stack([Es ** 3, Es ** 2, Es], axis=1)
    a3, a2, a1 = np.linalg.lstsq(V, exact, rcond=None)[0]
    assert abs(a3) < 1e-3 and abs(a2) < 1e-3
    printed = []
    for E in Es:
        c = oracle.error_constants_printed(E, nu)
        lam, mu = oracle.lame_2d(E, nu)
        printed.append(c[0] - (lam + 2 * mu) * c[5])
    p3, p2, p1 = np.linalg.lstsq(V, np.array(printed), rcond=None)[0]
    assert abs(p1 - a1) < 1e-3 * abs(a1)          # the linear parts agree
    assert abs(p2) > 0.5                           # the printed E^2 part does not vanish


def test_appendix_c_tau12_zeroes_printed_c5():
    for E, nu in ((0.3, 0.3), (0.11, 0.8), (1.0, 0.2)):
        lam, mu = oracle.lame_2d(E, nu)
        t12, t22 = oracle.fourth_order_taus(lam, mu)
        assert abs(oracle.error_constants_printed(E, nu, tau12=t12, tau22=t22)[4]) < 1e-15


def test_printed_correction_sign_increases_the_error():
    """Reading recorded in the design notes: with the printed D1, subtracting
    D1 dxx g (Eq. force_correction_x) doubles the longitudinal leading error
    of this scheme; adding it removes the D part."""
    E, nu = 0.3, 0.25
    lam, mu = oracle.lame_2d(E, nu)
    rates = oracle.relaxation_rates(lam, mu)
    D = oracle.error_constants_printed(E, nu)[5:]
    n = 256
    man = W.Manufactured(lam, mu, W._pw(n, n, [(1, 0, 1.0 + 0j, 0j)]))
    gx, gy = man.force()
    errs = {}
    for sign in (+1, -1):
        gxc, gyc = oracle.corrected_force_fd(gx, gy, sign * D)
        u = oracle.fields(F.steady_state_grid(gxc, gyc, rates), gxc, gyc, rates)[0]
        errs[sign] = float(np.max(np.abs(u - man.exact()[0])))
    base_u = oracle.fields(F.steady_state_grid(gx, gy, rates), gx, gy, rates)[0]
    base = float(np.max(np.abs(base_u - man.exact()[0])))
    assert errs[+1] > 1.5 * base and errs[-1] < 0.3 * base


def test_fd_correction_symbol():
    """Periodic central differences act on a plane wave by the exact symbols
    dxx -> 2 cos k1 - 2, dxy -> -sin k1 sin k2."""
    nx, ny = 24, 16
    pw = W._pw(nx, ny, [(3, 2, 1.0 + 0.5j, -0.3 + 0.2j)])
    gx, gy = pw.grid(pw.ax), pw.grid(pw.ay)
    D = (0.7, -0.4, 0.25)
    gxc, gyc = oracle.corrected_force_fd(gx, gy, D)
    k1, k2 = pw.k1[0], pw.k2[0]
    sxx, syy, sxy = 2 * np.cos(k1) - 2, 2 * np.cos(k2) - 2, -np.sin(k1) * np.sin(k2)
    ax, ay = pw.ax[0], pw.ay[0]
    ex = ax - (D[0] * sxx * ax + D[1] * sxy * ay + D[2] * syy * ax)
    ey = ay - (D[2] * sxx * ay + D[1] * sxy * ax + D[0] * syy * ay)
    assert np.max(np.abs(gxc - pw.grid(np.array([ex])))) < 1e-13
    assert np.max(np.abs(gyc - pw.grid(np.array([ey])))) < 1e-13


def test_library_constants_match_oracle_transcription():
    """Two independent transcriptions of Appendix B (C in the library, Python
    in the oracle) agree."""
    for E, nu, t12, t22 in ((0.3, 0.25, 0.5, 0.5), (0.11, 0.8, 1.2, 0.3), (1.0, -0.2, 0.7, 2.0)):
        lib = P.lbm_error_constants(E, nu, 1.0 / 3.0, t12, t22)
        ora = oracle.error_constants_printed(E, nu, tau12=t12, tau22=t22)
        assert np.max(np.abs(lib - ora)) < 1e-12 * max(1.0, np.max(np.abs(ora)))
