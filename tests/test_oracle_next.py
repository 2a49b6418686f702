"""Pins of the error-analysis helpers of Sec. 4 / Appendices B and C.

The oracle's transcription of the printed constants is compared with the
scheme's exact discrete leading error (per-mode closed form, extrapolated in
N), which pins the parts of Appendix B that are consistent with the scheme and
documents the parts that are not: three misprints (C2, D1, D2) and the sign
of the printed constants relative to the error equation as written."""
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
    """Reading of the printed D1: the exact longitudinal coefficient
    is linear in E~ (its E^2 and E^3 parts vanish), whereas the printed
    C1 - (mu + K) D1 keeps an E^2 term theta (nu - theta) tau12 E^2 / ((1 - theta^2)
    (1 - nu^2)^2) (1 - 1/(1 - nu^2)) that vanishes only at nu = 0 (the misprinted
    denominator of D1's E term, see error_constants_read)."""
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
    """Reading of the printed sign: with the printed D1, subtracting
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


# (E, nu, theta, tau12, tau22): standard and general rates, theta off 1/3, a
# negative Poisson ratio
EXTRACT_CASES = [(0.3, 0.25, 1 / 3, 0.5, 0.5), (0.11, 0.8, 1 / 3, 0.5, 0.5), (1.0, 0.3, 1 / 3, 0.5, 0.5),
                 (0.3, 0.0, 1 / 3, 0.9, 0.5), (0.05, 0.6, 1 / 3, 0.7, 0.3), (0.2, 0.7, 0.5, 0.8, 0.4),
                 (0.3, 0.25, 0.25, 0.5, 1.5), (0.3, 0.4, 0.6, 0.5, 0.5), (1.0, -0.2, 1 / 3, 0.7, 2.0)]


def _close(a, b, scale):
    return abs(a - b) <= 1e-4 * scale + 1e-6


@pytest.mark.parametrize("E,nu,th,t12,t22", EXTRACT_CASES)
def test_exact_leading_error_structure(E, nu, th, t12, t22):
    """The scheme's leading error has the structure of Eq. ux_order2 and its
    y twin: the over-determined relations of the extraction (C2 + C4 from the
    decay rates and from the eigenvector tilts; the E3 and E4 steady-state
    combinations) hold to the extrapolation error."""
    ex, checks = oracle.leading_error_exact(E, nu, theta=th, tau12=t12, tau22=t22)
    scale = float(np.max(np.abs(ex)))
    for name, v in checks.items():
        assert abs(v) <= 1e-4 * scale + 1e-6, (name, v)


@pytest.mark.parametrize("E,nu,th,t12,t22", EXTRACT_CASES)
def test_printed_constants_against_the_scheme(E, nu, th, t12, t22):
    """C1, C3, C4, C5 and D3 as printed are the scheme's; C2, D1 and D2 are
    the scheme's once the three misprints are read (error_constants_read);
    as printed, C2 differs at every point and D1, D2 wherever
    theta (nu - theta) resp. q is non-zero off nu = 0."""
    ex, _ = oracle.leading_error_exact(E, nu, theta=th, tau12=t12, tau22=t22)
    pr = oracle.error_constants_printed(E, nu, theta=th, tau12=t12, tau22=t22)
    rd = oracle.error_constants_read(E, nu, theta=th, tau12=t12, tau22=t22)
    scale = float(np.max(np.abs(ex)))
    for i in (0, 2, 3, 4, 7):
        assert _close(pr[i], ex[i], scale), ("printed", i, pr[i], ex[i])
    for i in range(8):
        assert _close(rd[i], ex[i], scale), ("read", i, rd[i], ex[i])
    assert not _close(pr[1], ex[1], scale)
    if nu != 0.0:
        q = th * th * (1 + nu) + nu - 2 * th - 1
        assert _close(pr[5], ex[5], scale) == (abs(th * (nu - th) * t12 * E) < 1e-12)
        assert not _close(pr[6], ex[6], scale) or abs(q) < 1e-12
    else:
        assert _close(pr[5], ex[5], scale) and _close(pr[6], ex[6], scale)


@pytest.mark.parametrize("E,nu,th,t12,t22", EXTRACT_CASES[::2])
def test_extracted_constants_predict_another_angle(E, nu, th, t12, t22):
    """Out-of-sample check of Eq. ux_order2's structure: the constants
    extracted at phi = 0, 45 degrees and atan(1/2) predict, at tan(phi) = 1/3,
    the O(k^4) decay rates and O(k^2) displacement tilts of free plane waves and
    the O(k^4) steady-state error under a force, as computed from the one-step
    operator directly."""
    ex, _ = oracle.leading_error_exact(E, nu, theta=th, tau12=t12, tau22=t22)
    C1, C2, C3, C4, C5, D1, D2, D3 = ex
    lam, mu = oracle.lame_2d(E, nu)
    K = lam + mu
    rates = oracle.relaxation_rates(lam, mu, theta=th, tau12=t12, tau22=t22)
    phi = np.arctan(1.0 / 3.0)
    c, s = np.cos(phi), np.sin(phi)
    vL, vT = np.array([c, s]), np.array([-s, c])
    Mm = F.moment_matrix()
    sigma = -1.0

    def measured(kap):
        w, V = np.linalg.eig(F.amplification_matrix(rates, kap * c, kap * s))
        out = {}
        for j in np.argsort(-np.abs(w))[:2]:
            U = Mm[:2] @ V[:, j]
            kind = "L" if abs(np.vdot(vL, U)) > abs(np.vdot(vT, U)) else "T"
            own, other = (vL, vT) if kind == "L" else (vT, vL)
            s2 = (mu + K) if kind == "L" else mu
            out[kind] = ((np.log(w[j]).real + s2 * kap ** 2) / kap ** 4,
                         (np.vdot(other, U) / np.vdot(own, U)).real / kap ** 2)
        return out

    a, b = measured(0.01), measured(0.02)
    got = {k: [(4 * a[k][i] - b[k][i]) / 3 for i in range(2)] for k in ("L", "T")}
    c6s6, c2s2, g = c ** 6 + s ** 6, c * c * s * s, c * s * (c * c - s * s)
    want = {"L": [sigma * (C1 * c6s6 + (C2 + C3 + C4 + C5) * c2s2), sigma * g * (C5 - C1 + C4) / (-K)],
            "T": [sigma * (C5 * c6s6 + (C1 + C3 - C2 - C4) * c2s2), sigma * g * (C5 - C1 + C2) / K]}
    scale = float(np.max(np.abs(ex)))
    for k in ("L", "T"):
        for i in range(2):
            assert abs(got[k][i] - want[k][i]) <= 1e-4 * scale / (1.0 if i == 0 else min(K, mu)) + 1e-6, \
                (k, i, got[k][i], want[k][i])

    # steady state under a force: (U - U0) = sigma M^-1 (A - Dm M) U0 at O(k^4)
    A = F.operator(rates)
    Bx, By = F.force_vectors(rates)

    def steady(kap):
        kx, ky = kap * c, kap * s
        Mk = np.array([[mu * kap ** 2 + K * kx * kx, K * kx * ky], [K * kx * ky, mu * kap ** 2 + K * ky * ky]])
        S = F.shift_diag(kx, ky)
        cols = []
        for U0 in (np.array([1.0, 0.0]), np.array([0.0, 1.0])):
            gh = Mk @ U0
            fh = np.linalg.solve(np.eye(8) - S[:, None] * A, S * (Bx * gh[0] + By * gh[1]))
            U = Mm[:2] @ fh + 0.5 * gh
            cols.append(sigma * (Mk @ (U - U0)).real / kap ** 4)
        return np.stack(cols, axis=1)

    Q = (4 * steady(0.01) - steady(0.02)) / 3
    Am = np.array([[C1 * c ** 4 + C3 * c2s2 + C5 * s ** 4, C2 * c ** 3 * s + C4 * c * s ** 3],
                   [C2 * c * s ** 3 + C4 * c ** 3 * s, C1 * s ** 4 + C3 * c2s2 + C5 * c ** 4]])
    Dm = np.array([[D1 * c * c + D3 * s * s, D2 * c * s], [D2 * c * s, D3 * c * c + D1 * s * s]])
    Mh = np.array([[mu + K * c * c, K * c * s], [K * c * s, mu + K * s * s]])
    assert np.max(np.abs(Q - (Am - Dm @ Mh))) <= 1e-4 * scale + 1e-6


def test_exact_leading_error_matches_axis_modes():
    """The general extraction agrees with the axis-mode steady states of
    leading_error_axis (one lattice of 2048^2, not extrapolated: agreement to
    its O(N^-2) remainder): E1 = C1 - (mu + K) D1 and E5 = C5 - mu D3."""
    for E, nu in ((0.3, 0.25), (0.11, 0.8)):
        ex, _ = oracle.leading_error_exact(E, nu)
        lam, mu = oracle.lame_2d(E, nu)
        a1, a5 = oracle.leading_error_axis(E, nu)
        assert abs(-a1 - (ex[0] - (lam + 2 * mu) * ex[5])) < 5e-4 * abs(a1) + 1e-6
        assert abs(-a5 - (ex[4] - mu * ex[7])) < 5e-4 * abs(a5) + 1e-6


def test_improved_scheme_reduces_the_error_tenfold():
    """Sec. 6.3.2: with the force correction of Eqs. force_correction_x/y the
    paper reports errors about one order of magnitude below the standard
    scheme (nu = 0.8; E = 0.11 standard, E = 0.085 improved; the field of
    Sec. 6.3.1).  With the read D1..D3, applied with the sign of the error
    equation (g' = g + D-terms, reading of the printed sign), the exact steady
    states show it; with the printed D1..D3 (either sign) at most 1.9x."""
    def err(E, n, D=None):
        lam, mu = oracle.lame_2d(E, 0.8)
        rates = oracle.relaxation_rates(lam, mu)
        man = W.paper_field(n, lam, mu)
        gx, gy = man.force()
        if D is not None:
            gx, gy = oracle.corrected_force_fd(gx, gy, D)
        u = oracle.fields(F.steady_state_grid(gx, gy, rates), gx, gy, rates)[:2]
        ue = man.exact()[:2]
        return float(np.max(np.abs(u - ue)) / np.max(np.abs(ue)))
    D_read = oracle.error_constants_read(0.085, 0.8)[5:]
    D_printed = oracle.error_constants_printed(0.085, 0.8)[5:]
    for n in (40, 80):
        standard = err(0.11, n)
        improved = err(0.085, n, -D_read)
        assert standard / improved > 7.0, (n, standard, improved)
        for d in (D_printed, -D_printed):
            assert standard / err(0.085, n, d) < 2.0


def test_library_scheme_constants_match_the_scheme():
    """lbm_error_constants_scheme (C, library) equals the oracle's read
    constants and the exact discrete extraction; the cancelling correction
    d = -(D1, D2, D3) is what the improved-scheme test uses."""
    for E, nu, th, t12, t22 in EXTRACT_CASES[:6]:
        lib = P.lbm_error_constants_scheme(E, nu, th, t12, t22)
        rd = oracle.error_constants_read(E, nu, theta=th, tau12=t12, tau22=t22)
        assert np.max(np.abs(lib - rd)) < 1e-12 * max(1.0, np.max(np.abs(rd)))
        ex, _ = oracle.leading_error_exact(E, nu, theta=th, tau12=t12, tau22=t22)
        assert np.max(np.abs(lib - ex)) <= 1e-4 * np.max(np.abs(ex)) + 1e-6
    with pytest.raises(P.LBMError):
        P.lbm_error_constants_scheme(-1.0, 0.3)


@pytest.mark.parametrize("E,nu", [(0.11, 0.8), (0.2, 0.5)])
def test_fourth_order_special_case(E, nu):
    """Sec. 6.3.3: for a displacement field without mixed fourth derivatives
    only C1 and C5 drive the leading error; with tau12 from Appendix C (zeroes
    C5), tau22 zeroing C1, and the force correction d = -(D1, D2, D3), the
    exact steady states converge at fourth order (the paper reports 4.00).
    Appendix C's printed tau22 leaves second order."""
    lam, mu = oracle.lame_2d(E, nu)
    t12, t22 = oracle.fourth_order_taus_scheme(lam, mu)
    _, t22_printed = oracle.fourth_order_taus(lam, mu)

    def errors(tau22):
        rates = oracle.relaxation_rates(lam, mu, tau12=t12, tau22=tau22)
        D = oracle.error_constants_read(E, nu, tau12=t12, tau22=tau22)[5:]
        out = []
        for n in (32, 64, 128):
            man = W.fourth_order_field(n, lam, mu)
            gx, gy = oracle.corrected_force_fd(*man.force(), -D)
            u = oracle.fields(F.steady_state_grid(gx, gy, rates), gx, gy, rates)[:2]
            ue = man.exact()[:2]
            out.append(float(np.max(np.abs(u - ue)) / np.max(np.abs(ue))))
        return np.log2(np.array(out[:-1]) / np.array(out[1:]))
    assert F.spectral_radius(oracle.relaxation_rates(lam, mu, tau12=t12, tau22=t22)) <= 1.0 + 1e-12
    assert np.all(errors(t22) > 3.9)
    assert np.all(errors(t22_printed) < 2.2)


def test_library_fourth_order_taus_match_oracle():
    for E, nu in ((0.11, 0.8), (0.2, 0.5), (0.3, 0.3)):
        lam, mu = oracle.lame_2d(E, nu)
        want = oracle.fourth_order_taus_scheme(lam, mu)
        got = P.lbm_fourth_order_taus(E, nu)
        assert np.allclose(got, want, rtol=1e-12, atol=0.0)
        c = oracle.error_constants_read(E, nu, tau12=got[0], tau22=got[1])
        assert abs(c[0]) < 1e-14 and abs(c[4]) < 1e-14
    with pytest.raises(P.LBMError):
        P.lbm_fourth_order_taus(0.3, 1.0 / 3.0)


def test_library_constants_match_oracle_transcription():
    """Two independent transcriptions of Appendix B (C in the library, Python
    in the oracle) agree."""
    for E, nu, t12, t22 in ((0.3, 0.25, 0.5, 0.5), (0.11, 0.8, 1.2, 0.3), (1.0, -0.2, 0.7, 2.0)):
        lib = P.lbm_error_constants(E, nu, 1.0 / 3.0, t12, t22)
        ora = oracle.error_constants_printed(E, nu, tau12=t12, tau22=t22)
        assert np.max(np.abs(lib - ora)) < 1e-12 * max(1.0, np.max(np.abs(ora)))
