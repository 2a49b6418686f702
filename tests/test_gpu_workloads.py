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
