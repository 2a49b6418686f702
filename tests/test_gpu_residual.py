"""The steady-state residual of every storage type against the oracle.

The stopping test of Sec. 2.1 (reading: r_inf = max|u^t - u^(t-k)| /
(k max|u^t|) and its L2 analogue) is what decides when a solve is done.  The
library evaluates it from the state the check step reads: FP64 storage in
FP64, FP32 and FP16-shifted storage from an exact FP32-pair evaluation of
u = mbar_10 = m_10 + g_x / 2 (Table 2) of the FP32 pre-collision populations,
with a pair snapshot and FP64 partial sums.  Here the two states that a check
compares are exported (lbm_get_populations) from a second lattice that runs
the same steps, and oracle.residual of oracle.fields of those states (FP64,
with the force as the device holds it) must equal the library's report.

Tolerance.  The pair displacement is exact to about 2^-44 of the largest
partial sum of the moment butterfly (a few |u|), so du is known to about
2e-12 max|u| in absolute terms: |r - r_oracle| <= 1e-12 r + 2e-12 / k.  The
windows checked early in the run (u still growing, du ~ u) make the first
term dominate, i.e. 1e-12 relative; a window near steady state checks the
absolute term.  FP64 storage: the same bound (FP64 rounding of u).

Which state a check reads: the check rides on the last step of its window
(step index kj - 1) and measures that step's input state, the state after
kj - 1 steps.  FP32 storage gives the same bits on every launch plan, so the
exported states come from a one-step-per-launch lattice.  FP16-shifted
storage rounds to FP16 only where a launch ends: its one-step plan is
checked exactly; on the four-step wavefront the checked state is the FP32
state three steps into the launch, which is reproduced by the oracle from the
exported launch input (three FP64 steps against the kernel's three FP32
steps: the bound adds 3 x 2^-24 of the populations, 1e-6 / k absolute).
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2208_14870_gb300 as P  # noqa: E402
from paper_2208_14870_gb300 import Lattice  # noqa: E402


def device_force(gx, gy, dtype):
    """The force as the device stores it (FP32 for FP32 and FP16S storage)."""
    if dtype == "f64":
        return gx, gy
    return gx.astype(np.float32).astype(np.float64), gy.astype(np.float32).astype(np.float64)


def exported_states(nx, ny, lam, mu, dtype, gx, gy, marks, spl=1):
    """Populations after each number of steps in `marks` (ascending)."""
    out = []
    with Lattice(nx, ny, lam, mu, dtype) as lat:
        lat.steps_per_launch = spl
        lat.set_force(gx, gy)
        for m in marks:
            lat.iterate(m - lat.step)
            out.append(lat.populations())
    return out


def assert_residual(got, u_now, u_prev, k, abs_tol):
    r_inf, r_2 = oracle.residual(u_now, u_prev, k)
    umax = float(np.max(np.abs(u_now)))
    u2 = float(np.sqrt(np.sum(u_now * u_now)))
    assert abs(got[0] - r_inf) <= 1e-12 * r_inf + abs_tol, (got[0], r_inf)
    assert abs(got[1] - r_2) <= 1e-12 * r_2 + abs_tol, (got[1], r_2)
    assert abs(got[2] - umax) <= 1e-12 * umax
    assert abs(got[3] - u2) <= 1e-12 * u2
    assert got[4] == 0.0
    return r_inf


# (nx, ny, steps per launch): 48 x 40 runs one step per launch; 300 x 40
# runs the four-step wavefront (check on its last level) by default, or two
# steps per launch (check on the second step of a two-step tile launch)
PLANS = [(48, 40, 1), (300, 40, 4), (300, 40, 2), (300, 40, 1)]


@pytest.mark.parametrize("nx,ny,spl", PLANS)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("k,windows", [(10, 2), (100, 25)])
def test_residual_matches_oracle(dtype, nx, ny, spl, k, windows):
    if dtype == "f64" and spl > 1:
        pytest.skip("FP64 storage runs one step per launch")
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    pw = W.random_force(nx, ny, 8, 4, seed=nx + 7 * k)
    gx, gy = W.random_force_grid(pw)
    with Lattice(nx, ny, lam, mu, dtype) as lat:
        lat.steps_per_launch = spl
        lat.set_force(gx, gy)
        got = lat.iterate_checked(k * windows, k)
    n = k * windows
    fa, fb = exported_states(nx, ny, lam, mu, dtype, gx, gy, [n - k - 1, n - 1])
    dgx, dgy = device_force(gx, gy, dtype)
    ua = oracle.fields(fa, dgx, dgy, rates)[:2]
    ub = oracle.fields(fb, dgx, dgy, rates)[:2]
    r = assert_residual(got, ub, ua, k, 2e-12 / k)
    print("%s %dx%d spl=%d k=%d after %d steps: r_inf %.6e (device %.6e)" % (
        dtype, nx, ny, spl, k, n, r, got[0]))


@pytest.mark.parametrize("k,windows", [(10, 2), (100, 25)])
def test_f16s_residual_one_step_plan_matches_oracle(k, windows):
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    nx, ny = 300, 40
    pw = W.random_force(nx, ny, 8, 4, seed=3 + k)
    gx, gy = W.random_force_grid(pw)
    with Lattice(nx, ny, lam, mu, "f16s") as lat:
        lat.steps_per_launch = 1
        lat.set_force(gx, gy)
        got = lat.iterate_checked(k * windows, k)
    n = k * windows
    fa, fb = exported_states(nx, ny, lam, mu, "f16s", gx, gy, [n - k - 1, n - 1], spl=1)
    dgx, dgy = device_force(gx, gy, "f16s")
    ua = oracle.fields(fa, dgx, dgy, rates)[:2]
    ub = oracle.fields(fb, dgx, dgy, rates)[:2]
    assert_residual(got, ub, ua, k, 2e-12 / k)


@pytest.mark.parametrize("k,windows", [(12, 2), (100, 25)])
def test_f16s_residual_on_the_wavefront(k, windows):
    """Windows of 12 (100) steps on the four-step wavefront: 8 (96) plain
    steps, then the checked launch of four steps whose last level reads the
    FP32 state after three of them."""
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    nx, ny = 300, 40
    pw = W.random_force(nx, ny, 8, 4, seed=5 + k)
    gx, gy = W.random_force_grid(pw)
    n = k * windows
    with Lattice(nx, ny, lam, mu, "f16s") as lat:
        assert lat.steps_per_launch == 4
        lat.set_force(gx, gy)
        got = lat.iterate_checked(n, k)
    # the launch inputs of the last two checked launches (steps kj - 4), from
    # a lattice on the same launch plan (iterate_checked with the same windows)
    states = []
    for m in (n - k - 4, n - 4):
        with Lattice(nx, ny, lam, mu, "f16s") as lat:
            lat.set_force(gx, gy)
            lat.iterate_checked(m - m % k, k)
            lat.iterate(m % k)
            states.append(lat.populations())
    dgx, dgy = device_force(gx, gy, "f16s")
    us = [oracle.fields(oracle.run(f, dgx, dgy, rates, 3), dgx, dgy, rates)[:2] for f in states]
    r_inf, r_2 = oracle.residual(us[1], us[0], k)
    tol = 1e-6 / k
    assert abs(got[0] - r_inf) <= 1e-12 * r_inf + tol, (got[0], r_inf)
    assert abs(got[1] - r_2) <= 1e-12 * r_2 + tol, (got[1], r_2)
    print("f16s wavefront k=%d: r_inf %.6e (device %.6e)" % (k, r_inf, got[0]))


def _served_request(index):
    """Request `index` of the seeded serving stream's requests with sides up to
    2048 (the benchmark's served prefix)."""
    reqs = [r for r in W.served_requests(rate_hz=20.0) if max(r.nx, r.ny) <= 2048]
    return reqs[index]


@pytest.mark.parametrize("index", [23, 74])
def test_fp16s_windows_stretch_past_the_rounding_floor(index):
    """Elongated FP16S requests of the serving stream (100 x 884, nu = 0.39;
    1311 x 64, nu = 0.23): their rounding floor follows the shorter side, and a
    window sized by the longer one never got below tol 1e-8.  With windows
    sized by the shorter side and doubled while the residual stagnates,
    lbm_solve and the batch arena both converge within a few times the steps
    the slowest mode needs."""
    import math
    r = _served_request(index)
    assert r.dtype == "f16s"
    ks = [(int(a), int(b)) for a, b in zip(r.force.kx, r.force.ky)]
    kk = min((2 * math.pi * kx / r.nx) ** 2 + (2 * math.pi * ky / r.ny) ** 2 for kx, ky in ks)
    expect = math.log(r.mu * kk / 1e-8) / (r.mu * kk)
    gx, gy = W.random_force_grid(r.force)
    with Lattice(r.nx, r.ny, r.lam, r.mu, "f16s") as lat:
        lat.set_force(gx, gy)
        st, iters, res = lat.solve(1e-8, int(20 * expect), 100)
    assert st == P.LBM_OK and res < 1e-8, (st, iters, res)
    assert iters < 6 * expect, (iters, expect)
    results, _ = P.batch_solve([(r.nx, r.ny, r.lam, r.mu, gx, gy)], dtype="f16s", tol=1e-8, check_every=100,
                               max_iters=int(20 * expect), fields=False)
    assert results[0]["status"] == P.LBM_OK and results[0]["iters"] < 6 * expect, results[0]
    print("request %d %dx%d: lbm_solve %d steps, batch %d (slowest mode needs ~%.0f)" % (
        index, r.nx, r.ny, iters, results[0]["iters"], expect))
