"""Second workload (Gaussian hill, Sec. 6.3.5) through the CUDA path, and the
stability warning of the binding."""
import numpy as np
import pytest

import oracle
import oracle.fourier as F
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2208_14870_gb300 as P  # noqa: E402


@pytest.mark.parametrize("dtype,tol,rtol", [("f64", 1e-13, 1e-10), ("f32", 2e-9, 2e-5), ("f16s", 2e-7, 2e-3)])
def test_gaussian_hill_steady_state(dtype, tol, rtol):
    n = 96
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    gx, gy, ex = W.gaussian_hill(n, lam, mu)
    fix = oracle.fields(F.steady_state_grid(gx, gy, rates), gx, gy, rates)
    with P.Lattice(n, n, lam, mu, dtype) as lat:
        lat.set_force(gx, gy)
        st, iters, r = lat.solve(tol, 5_000_000, 200)
        assert st == P.LBM_OK
        got = lat.fields()
    eu = np.max(np.abs(got[:2] - fix[:2])) / np.max(np.abs(fix[:2]))
    es = np.max(np.abs(got[2:] - fix[2:])) / np.max(np.abs(fix[2:]))
    assert eu < rtol and es < rtol, (eu, es)


def test_unstable_parameters_warn():
    lam, mu = W.lame_2d(0.082, -0.4)
    with pytest.warns(RuntimeWarning, match="unstable"):
        lat = P.Lattice(16, 16, lam, mu, "f32", check_stability=True)
    lat.close()
    lam, mu = W.lame_2d(1.0, 0.3)
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        P.Lattice(16, 16, lam, mu, "f32", check_stability=True).close()


def _paper_case(E, nu, n, field, taus=None, correct=False):
    """FP64 steady state of a manufactured field through the C ABI (standard,
    corrected force, general tau12/tau22), checked against the oracle's exact
    fixed point of the same (corrected) force; returns the relative Linf
    displacement error against the analytical field."""
    lam, mu = W.lame_2d(E, nu)
    t12, t22 = taus if taus is not None else (0.5, 0.5)
    rates = oracle.relaxation_rates(lam, mu, tau12=t12, tau22=t22)
    man = field(n, lam, mu)
    gx, gy = man.force()
    kw = dict(tau12=t12, tau22=t22) if taus is not None else {}
    with P.Lattice(n, n, lam, mu, "f64", **kw) as lat:
        if correct:
            d = -P.lbm_error_constants_scheme(E, nu, 0.0, t12, t22)[5:]
            lat.set_force_corrected(gx, gy, d)
            gx, gy = oracle.corrected_force_fd(gx, gy, d)
        else:
            lat.set_force(gx, gy)
        st, iters, r = lat.solve(1e-14, 10_000_000, 200)
        assert st == P.LBM_OK
        got = lat.fields()[:2]
    fix = oracle.fields(F.steady_state_grid(gx, gy, rates), gx, gy, rates)[:2]
    assert np.max(np.abs(got - fix)) < 1e-9 * np.max(np.abs(fix))
    ue = man.exact()[:2]
    return float(np.max(np.abs(got - ue)) / np.max(np.abs(ue)))


def test_improved_scheme_on_the_device():
    """Sec. 6.3.2 through the C ABI: the force correction with
    d = -(D1, D2, D3) of lbm_error_constants_scheme at nu = 0.8, E = 0.085
    gives errors about eight times below the standard scheme at E = 0.11."""
    standard = _paper_case(0.11, 0.8, 40, W.paper_field)
    improved = _paper_case(0.085, 0.8, 40, W.paper_field, correct=True)
    assert standard / improved > 7.0, (standard, improved)


def test_fourth_order_case_on_the_device():
    """Sec. 6.3.3 through the C ABI: lbm_fourth_order_taus (C5 = C1 = 0) and the
    corrected force give fourth-order convergence for the field without mixed
    fourth derivatives."""
    E, nu = 0.11, 0.8
    taus = P.lbm_fourth_order_taus(E, nu)
    e = [_paper_case(E, nu, n, W.fourth_order_field, taus=taus, correct=True) for n in (32, 64)]
    assert np.log2(e[0] / e[1]) > 3.8, e
