"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: the matrix printed
in Sec. 4, the numbers printed in Sec. 6, the exact solution of the target PDE
(second-order convergence), brute-force dense operators on tiny lattices built
with library routines, and exact invariants (conservation, symmetry,
translation equivariance, linearity, inertness of the rest population).
"""
import os

import numpy as np
import pytest

import oracle
import oracle.fourier as F
import workloads as W
from conftest import GOLDEN

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def printed_M():
    return np.loadtxt(os.path.join(GOLDEN, "moment_matrix.txt"))


# Velocity table of the paper's population table (Sec. 4), typed here
# independently of the oracle.
CX = [1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 1, 0, -1, 1, 1, -1, -1]


def rates_E_nu(E, nu, **kw):
    lam, mu = oracle.lame_2d(E, nu)
    return oracle.relaxation_rates(lam, mu, **kw)


# ---------------------------------------------------------------------------
# Moment transform and its inverse
# ---------------------------------------------------------------------------

def test_moment_matrix_is_the_printed_one():
    """Sec. 4 prints M; the oracle's moments of unit populations are its columns."""
    M = printed_M()
    assert np.array_equal(F.moment_matrix(), M)
    for p in range(8):
        f = np.zeros((8, 1, 1))
        f[p] = 1.0
        assert np.array_equal(oracle.moments(f)[:, 0, 0], M[:, p])


def test_back_transformation_inverts_raw_moments():
    """Eq. moments_post: the oracle's solve of the raw-moment system is the
    inverse of the raw-moment matrix (built here from the definition, Eq. moments)."""
    ma = [1, 0, 1, 2, 0, 1, 2, 2]
    mb = [0, 1, 1, 0, 2, 2, 1, 2]
    T = np.array([[CX[p] ** ma[r] * CY[p] ** mb[r] for p in range(8)] for r in range(8)], float)
    inv = oracle.raw_moment_inverse(8)
    assert np.allclose(inv @ T, np.eye(8), atol=1e-15)
    assert np.allclose(inv, np.linalg.inv(T), atol=1e-15)


def test_no_relaxation_no_force_is_identity_collision():
    """With every rate 0 and g = 0, Eq. collision leaves all moments unchanged,
    so collide(f) = f and one step is a pure shift of each population by c_i."""
    f = W.random_populations(8, 5, 3, seed=1)
    z = np.zeros((3, 5))
    w = np.array([0, 0, 0, 0, 0, 0, 1 / 3.0])
    assert np.allclose(oracle.collide(f, z, z, w), f, atol=1e-15)
    out = oracle.run(f, z, z, w, 1)
    for p in range(8):
        assert np.allclose(out[p], np.roll(f[p], shift=(CY[p], CX[p]), axis=(0, 1)), atol=1e-15)


# ---------------------------------------------------------------------------
# One step against the dense operator of Eq. lbmvector (4 x 4 lattice)
# ---------------------------------------------------------------------------

def dense_step_matrix(nx, ny, rates):
    """128 x 128 (for 4 x 4) one-step matrix and force matrix, assembled from the
    printed M (Sec. 4), numpy's inverse, Lambda, the Table 1 equilibria and the
    streaming permutation of Eq. streaming."""
    w11, ws, wd, w12, w21, w22, th = rates
    M = printed_M()
    Minv = np.linalg.inv(M)
    Lam = np.diag([0, 0, w11, ws, wd, w12, w21, w22])
    Meq = np.zeros((8, 8))
    Meq[0], Meq[1] = M[0], M[1]
    Meq[5], Meq[6] = th * M[0], th * M[1]          # Table 1: m12eq = theta*m10
    A = Minv @ Lam @ Meq + Minv @ (np.eye(8) - Lam) @ M
    ex = np.zeros(8); ex[0] = 1.0; ex[5] = w12 * th / 2      # m10* += g, m12eq += theta g/2
    ey = np.zeros(8); ey[1] = 1.0; ey[6] = w21 * th / 2
    Bx, By = Minv @ ex, Minv @ ey
    n = nx * ny
    big = np.zeros((8 * n, 8 * n))
    bgx = np.zeros((8 * n, n))
    bgy = np.zeros((8 * n, n))
    for y in range(ny):
        for x in range(nx):
            s = y * nx + x
            for p in range(8):
                d = ((y + CY[p]) % ny) * nx + (x + CX[p]) % nx
                big[p * n + d, [l * n + s for l in range(8)]] = A[p]
                bgx[p * n + d, s] = Bx[p]
                bgy[p * n + d, s] = By[p]
    return big, bgx, bgy


@pytest.mark.parametrize("nu,E", [(0.3, 1.0), (0.8, 0.11), (-0.2, 0.5)])
def test_single_step_matches_dense_operator_4x4(nu, E):
    nx = ny = 4
    rates = rates_E_nu(E, nu)
    f = W.random_populations(8, nx, ny, seed=7)
    gx = W.random_field(nx, ny, seed=8)
    gy = W.random_field(nx, ny, seed=9)
    big, bgx, bgy = dense_step_matrix(nx, ny, rates)
    ref = big @ f.reshape(-1) + bgx @ gx.reshape(-1) + bgy @ gy.reshape(-1)
    out = oracle.run(f, gx, gy, rates, 1)
    assert np.max(np.abs(out.reshape(-1) - ref)) < 1e-14 * max(1.0, np.max(np.abs(ref)))


def test_general_higher_order_rates_match_dense_operator():
    """w_12 = w_21 != 1 and w_22 != 1 (used by the fourth-order case, App. C)."""
    rates = rates_E_nu(0.7, 0.25, tau12=0.9, tau22=0.3)
    f = W.random_populations(8, 3, 4, seed=11)
    gx = W.random_field(3, 4, seed=12)
    gy = W.random_field(3, 4, seed=13)
    big, bgx, bgy = dense_step_matrix(3, 4, rates)
    ref = big @ f.reshape(-1) + bgx @ gx.reshape(-1) + bgy @ gy.reshape(-1)
    out = oracle.run(f, gx, gy, rates, 1)
    assert np.max(np.abs(out.reshape(-1) - ref)) < 1e-14


# ---------------------------------------------------------------------------
# Exact invariants
# ---------------------------------------------------------------------------

def test_first_moment_balance_per_step():
    """Sum over nodes of m_10 grows by exactly sum(g_x) per step (Eqs. coll10 and
    coll10post; streaming only moves populations)."""
    nx, ny = 7, 5
    rates = rates_E_nu(1.0, 0.3)
    f = W.random_populations(8, nx, ny, seed=3)
    gx = W.random_field(nx, ny, seed=4)
    gy = W.random_field(nx, ny, seed=5)
    m0 = oracle.moments(f)
    m1 = oracle.moments(oracle.run(f, gx, gy, rates, 1))
    assert abs(m1[0].sum() - m0[0].sum() - gx.sum()) < 1e-12
    assert abs(m1[1].sum() - m0[1].sum() - gy.sum()) < 1e-12


def test_zero_force_keeps_zero_state():
    rates = rates_E_nu(1.0, 0.3)
    z = np.zeros((6, 9))
    out = oracle.run(oracle.zero_state(9, 6), z, z, rates, 17)
    assert not np.any(out)


def test_translation_equivariance():
    """Shifting f and g by whole nodes shifts the result (periodic wrap, Sec. 5.1)."""
    nx, ny = 6, 5
    rates = rates_E_nu(0.9, 0.1)
    f = W.random_populations(8, nx, ny, seed=21)
    gx = W.random_field(nx, ny, seed=22)
    gy = W.random_field(nx, ny, seed=23)
    sh = (2, 3)
    a = np.roll(oracle.run(f, gx, gy, rates, 3), shift=sh, axis=(1, 2))
    b = oracle.run(np.roll(f, sh, axis=(1, 2)), np.roll(gx, sh, axis=(0, 1)),
                   np.roll(gy, sh, axis=(0, 1)), rates, 3)
    assert np.max(np.abs(a - b)) < 1e-14


def test_transpose_symmetry():
    """Swapping x and y maps populations (1 2)(3 4)(6 8), swaps g_x, g_y."""
    nx, ny = 5, 5
    perm = [1, 0, 3, 2, 4, 7, 6, 5]
    rates = rates_E_nu(1.0, 0.3)
    f = W.random_populations(8, nx, ny, seed=31)
    gx = W.random_field(nx, ny, seed=32)
    gy = W.random_field(nx, ny, seed=33)

    def tr(fa):
        out = np.empty_like(fa)
        for p in range(8):
            out[perm[p]] = fa[p].T
        return out

    a = tr(oracle.run(f, gx, gy, rates, 2))
    b = oracle.run(tr(f), gy.T.copy(), gx.T.copy(), rates, 2)
    assert np.max(np.abs(a - b)) < 1e-14
    fa = oracle.fields(f, gx, gy, rates)
    fb = oracle.fields(tr(f), gy.T.copy(), gx.T.copy(), rates)
    assert np.allclose(fa[0].T, fb[1]) and np.allclose(fa[2].T, fb[3]) and np.allclose(fa[4].T, fb[4])


def test_mirror_symmetry_x():
    """x -> -x maps populations (1 3)(5 6)(7 8), node n -> nx-1-n, g_x -> -g_x."""
    nx, ny = 6, 4
    perm = [2, 1, 0, 3, 5, 4, 7, 6]
    rates = rates_E_nu(0.6, 0.4)
    f = W.random_populations(8, nx, ny, seed=41)
    gx = W.random_field(nx, ny, seed=42)
    gy = W.random_field(nx, ny, seed=43)

    def mir(fa):
        out = np.empty_like(fa)
        for p in range(8):
            out[perm[p]] = fa[p][:, ::-1]
        return out

    a = mir(oracle.run(f, gx, gy, rates, 2))
    b = oracle.run(mir(f), -gx[:, ::-1].copy(), gy[:, ::-1].copy(), rates, 2)
    assert np.max(np.abs(a - b)) < 1e-14


def test_linearity():
    nx, ny = 4, 6
    rates = rates_E_nu(1.0, 0.2)
    f1 = W.random_populations(8, nx, ny, seed=51)
    f2 = W.random_populations(8, nx, ny, seed=52)
    g = [W.random_field(nx, ny, seed=s) for s in (53, 54, 55, 56)]
    a, b = 0.75, -1.5
    lhs = oracle.run(a * f1 + b * f2, a * g[0] + b * g[2], a * g[1] + b * g[3], rates, 3)
    rhs = a * oracle.run(f1, g[0], g[1], rates, 3) + b * oracle.run(f2, g[2], g[3], rates, 3)
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_rest_population_is_inert():
    """D2Q9 with the rest population f_00 gives the same D2Q8 populations and
    fields (Sec. 3.3.2: m_00 does not influence the scheme; D2Q8 suffices)."""
    nx, ny = 5, 4
    rates = rates_E_nu(1.0, 0.3)
    f9 = W.random_populations(9, nx, ny, seed=61)
    gx = W.random_field(nx, ny, seed=62)
    gy = W.random_field(nx, ny, seed=63)
    o9 = oracle.run(f9, gx, gy, rates, 4)
    o8 = oracle.run(np.ascontiguousarray(f9[:8]), gx, gy, rates, 4)
    assert np.max(np.abs(o9[:8] - o8)) < 1e-13
    assert np.max(np.abs(oracle.fields(o9, gx, gy, rates) - oracle.fields(o8, gx, gy, rates))) < 1e-13
    # m_00 is carried unchanged in total (not collided, streaming conserves it)
    assert abs(oracle.moments(o9)[8].sum() - oracle.moments(f9)[8].sum()) < 1e-12


# ---------------------------------------------------------------------------
# Steady state: exact discrete closed form, time stepping, continuum limit
# ---------------------------------------------------------------------------

def test_time_stepping_reaches_exact_discrete_steady_state():
    """The C oracle iterated to a tight residual equals the per-mode closed form
    (two independent computations of the same discrete fixed point)."""
    nx, ny = 16, 12
    rates = rates_E_nu(1.0, 0.3)
    pw = W.random_force(nx, ny, n_modes=4, kmax=3, seed=99)
    gx, gy = W.random_force_grid(pw)
    f, it, r = oracle.solve(gx, gy, rates, tol=1e-14, check_every=100)
    fss = F.steady_state_grid(gx, gy, rates)
    assert np.max(np.abs(f - fss)) < 1e-11 * np.max(np.abs(fss))
    # the per-mode evaluation agrees with the FFT-based one
    ks, fh, flh = F.steady_state_modes(nx, ny, pw.modes(), rates)
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    flm = np.stack([F.evaluate_modes(ks, flh[:, c], X, Y) for c in range(5)])
    assert np.max(np.abs(flm - oracle.fields(fss, gx, gy, rates))) < 1e-12 * np.max(np.abs(flm))


def _rel_errors(N, man, rates):
    gx, gy = man.force()
    fl = oracle.fields(F.steady_state_grid(gx, gy, rates), gx, gy, rates)
    ex = man.exact()
    dx = 1.0 / N
    # dimensionless stress = lattice stress / eps, eps = 1/N (Table 2)
    eu, es = fl[:2] - ex[:2], (fl[2:] - ex[2:]) * N
    nu2 = np.sqrt(dx * dx * np.sum(ex[:2] ** 2))
    ns2 = np.sqrt(dx * dx * np.sum((ex[2:] * N) ** 2))
    return np.array([np.sqrt(dx * dx * np.sum(eu ** 2)) / nu2, np.max(np.abs(eu)) / nu2,
                     np.sqrt(dx * dx * np.sum(es ** 2)) / ns2, np.max(np.abs(es)) / ns2])


def test_second_order_convergence_to_manufactured_solution():
    """Sec. 3.4 / Sec. 5: displacement and stress converge at second order to the
    exact solution of the target PDE (sweep field, E~ = 1, nu = 0.3)."""
    lam, mu = oracle.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    Ns = [32, 64, 128, 256]
    errs = np.array([_rel_errors(N, W.sinusoid(N, 1, lam, mu), rates) for N in Ns])
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(orders > 1.94) and np.all(orders < 2.06), orders


def test_paper_printed_accuracy_and_orders(printed):
    """Sec. 6.3.1: 3-4 % relative Linf displacement error at dx = 0.05 L and
    second-order slopes (printed 2.01 / 2.00 / 2.00 / 1.98) over 20^2 ... 100^2."""
    lam, mu = oracle.lame_2d(printed["standard_E"], printed["standard_nu"])
    rates = oracle.relaxation_rates(lam, mu)
    Ns = [20, 40, 60, 80, 100]
    errs = np.array([_rel_errors(N, W.paper_field(N, lam, mu), rates) for N in Ns])
    assert printed["standard_linf_rel_lo"] <= errs[0, 1] <= printed["standard_linf_rel_hi"]
    h = 1.0 / np.array(Ns)
    fit = [np.polyfit(np.log(h), np.log(errs[:, c]), 1)[0] for c in range(4)]
    want = [printed[k] for k in ("standard_order_l2_u", "standard_order_linf_u",
                                 "standard_order_l2_s", "standard_order_linf_s")]
    assert np.all(np.abs(np.array(fit) - np.array(want)) < 0.06), (fit, want)


def test_paper_steady_state_after_about_a_thousand_steps(printed):
    """Sec. 6.3.1: on the 20^2 mesh the steady state is reached after roughly
    10^3 steps: the Linf error is within 2 % of its limit at 10^3 steps and
    still more than 10 % away at 500."""
    lam, mu = oracle.lame_2d(printed["standard_E"], printed["standard_nu"])
    rates = oracle.relaxation_rates(lam, mu)
    N = int(printed["standard_n"])
    man = W.paper_field(N, lam, mu)
    gx, gy = man.force()
    ex = man.exact()
    nrm = np.sqrt(np.sum(ex[:2] ** 2) / N / N)
    final = np.max(np.abs(oracle.fields(F.steady_state_grid(gx, gy, rates), gx, gy, rates)[:2]
                          - ex[:2])) / nrm
    f500 = oracle.run(oracle.zero_state(N, N), gx, gy, rates, 500)
    f1000 = oracle.run(f500, gx, gy, rates, 500)
    e500 = np.max(np.abs(oracle.fields(f500, gx, gy, rates)[:2] - ex[:2])) / nrm
    e1000 = np.max(np.abs(oracle.fields(f1000, gx, gy, rates)[:2] - ex[:2])) / nrm
    assert abs(e1000 / final - 1) < 0.02
    assert abs(e500 / final - 1) > 0.10


def test_time_stepped_oracle_converges_to_pde_solution():
    """The C oracle itself (not only the closed form) converges at second order."""
    lam, mu = oracle.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    e = []
    for N in (32, 64):
        man = W.sinusoid(N, 1, lam, mu)
        gx, gy = man.force()
        f, it, r = oracle.solve(gx, gy, rates, tol=1e-12, check_every=100)
        fl = oracle.fields(f, gx, gy, rates)
        e.append(np.max(np.abs(fl[:2] - man.exact()[:2])))
    assert 3.8 < e[0] / e[1] < 4.2


# ---------------------------------------------------------------------------
# Stability (Sec. 4, Sec. 6.3.5)
# ---------------------------------------------------------------------------

def test_declared_unstable_point_is_unstable_with_table1(printed):
    r = rates_E_nu(printed["unstable_E"], printed["unstable_nu"])
    assert F.spectral_radius(r) > 1.005


def test_printed_equilibrium_matrix_contradicts_section_6(printed):
    """The M^eq printed in Sec. 4 keeps the declared unstable point stable,
    which is why Table 1 is followed."""
    r = rates_E_nu(printed["unstable_E"], printed["unstable_nu"])
    assert F.spectral_radius(r, printed_meq=True) < 1 + 1e-9


def test_stable_range_of_poisson_ratios(printed):
    """Sec. 4: stable for nu in about [-0.3, 0.95] at a suitable E~; unstable
    again only for nu above about 0.996."""
    for nu in np.linspace(printed["stable_nu_lo"], printed["stable_nu_hi"], 6):
        assert F.spectral_radius(rates_E_nu(0.2, nu)) < 1 + 1e-9
    for E in (0.02, 0.05, 0.082, 0.11, 0.2, 0.5, 1.0):
        assert F.spectral_radius(rates_E_nu(E, 0.99)) < 1 + 1e-9
    assert max(F.spectral_radius(rates_E_nu(E, 0.999)) for E in (0.05, 0.082, 0.11)) > 1.005


def test_sweep_parameters_are_stable():
    """All Poisson ratios of the sweep at E~ = 1 (the configs' reading of E = 1)."""
    for nu in (0.0, 0.2, 0.3, 0.4, 0.45):
        assert F.spectral_radius(rates_E_nu(1.0, nu)) < 1 + 1e-9


def test_time_stepping_diverges_at_unstable_point(printed):
    """The growth predicted by the spectral radius shows up in the C oracle."""
    r = rates_E_nu(printed["unstable_E"], printed["unstable_nu"])
    f = W.random_populations(8, 16, 16, seed=5, scale=1e-6)
    z = np.zeros((16, 16))
    out = oracle.run(f, z, z, r, 1500)
    assert np.max(np.abs(out)) > 1e3 * np.max(np.abs(f))


# ---------------------------------------------------------------------------
# Host-side helpers of the oracle
# ---------------------------------------------------------------------------

def test_material_relations():
    lam, mu = oracle.lame_2d(1.0, 0.0)
    assert lam == 0.0 and mu == 0.5
    lam, mu = oracle.lame_2d(2.0, 0.5)
    assert abs((lam + mu) - 2.0 / (2 * (1 - 0.5))) < 1e-15   # K = E / (2 (1 - nu))


def test_theta_one_third_equalises_w11_and_wd():
    """Sec. 3.3.2: theta = 1/3 is the value for which tau_11 = tau_d."""
    for mu in (0.1, 0.385, 2.0):
        r = oracle.relaxation_rates(0.3, mu)
        assert abs(r[0] - r[2]) < 1e-15
    r = oracle.relaxation_rates(0.3, 0.4, theta=0.25)
    assert abs(r[0] - r[2]) > 1e-3


def test_residual_definition():
    u_prev = np.zeros((2, 3, 3))
    u_now = np.full((2, 3, 3), 2.0)
    u_now[0, 1, 1] = 4.0
    r_inf, r_2 = oracle.residual(u_now, u_prev, 10)
    assert abs(r_inf - 4.0 / (10 * 4.0)) < 1e-15 and abs(r_2 - 0.1) < 1e-15
    assert oracle.residual(np.zeros((2, 2, 2)), np.zeros((2, 2, 2)), 5) == (0.0, 0.0)


def test_grid_norms():
    e = np.ones((2, 4, 4))
    l2, linf = oracle.grid_norms(e, 0.25)
    assert abs(l2 - np.sqrt(0.0625 * 32)) < 1e-15 and linf == 1.0
