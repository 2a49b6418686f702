"""Continuous-batching server (lbm_server_*): results are the same alone and
in the mix, requests overlap on the device, admission respects the HBM
budget, and host-side faults (malformed or oversized requests, cancellation,
an unpolled consumer) are handled without touching the GPU's health."""
import threading
import time

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

GIB = 1 << 30


@pytest.fixture(autouse=True)
def _tune_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("LBM_AUTOTUNE_CACHE", str(tmp_path / "autotune.txt"))


def problem(nx, ny, nu, seed):
    lam, mu = W.lame_2d(1.0, nu)
    pw = W.random_force(nx, ny, 4, 3, seed=seed)
    gx, gy = W.random_force_grid(pw)
    return nx, ny, lam, mu, gx, gy, pw


def exact_fields(p):
    nx, ny, lam, mu, gx, gy, pw = p
    rates = oracle.relaxation_rates(lam, mu)
    ks, fh, flh = F.steady_state_modes(nx, ny, pw.modes(), rates)
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    return np.stack([F.evaluate_modes(ks, flh[:, c], X, Y) for c in range(5)])


def rel_per_field(a, b):
    """Displacement error relative to max |u| over both components, stress
    error relative to the largest stress component (a field that is tiny for a
    given force is not measured against its own maximum)."""
    eu = float(np.max(np.abs(a[:2] - b[:2]))) / max(float(np.max(np.abs(b[:2]))), 1e-300)
    es = float(np.max(np.abs(a[2:] - b[2:]))) / max(float(np.max(np.abs(b[2:]))), 1e-300)
    return max(eu, es)


# (nx, ny, solved transposed): 60 x 300 fits the arena better on its transpose
# (wavefront items instead of two-step tiles); its fields come back in the
# caller's orientation
@pytest.mark.parametrize("nx,ny,tr", [(96, 72, False), (60, 300, True)])
@pytest.mark.parametrize("dtype,tol,tol_fix", [("f32", 2e-9, 2e-5), ("f16s", 2e-7, 2e-3)])
def test_same_result_alone_and_in_the_mix(dtype, tol, tol_fix, nx, ny, tr):
    target = problem(nx, ny, 0.3, seed=42)
    with P.Server(2 * GIB, check_every=100) as srv:
        t = srv.submit(*target[:6], dtype=dtype, tol=tol)
        alone = srv.wait(t, 120.0)
        assert alone["status"] == P.LBM_OK
        assert alone["transposed"] == tr
        assert alone["fields"].shape == (5, ny, nx)
        assert srv.stats()["peak_running"] == 1
    others = [problem(int(s), int(s * 0.75) + 3, 0.05 * i, seed=100 + i)
              for i, s in enumerate([40, 200, 64, 150, 32, 128, 90, 250, 48, 180])]
    with P.Server(2 * GIB, check_every=100) as srv:
        tickets = []

        def feeder():
            for i, p in enumerate(others):
                f32 = i % 2 == 1
                tickets.append((i, srv.submit(*p[:6], dtype="f32" if f32 else "f16s",
                                              tol=2e-9 if f32 else 2e-7)))
                time.sleep(0.01)

        th = threading.Thread(target=feeder)
        th.start()
        time.sleep(0.02)
        tt = srv.submit(*target[:6], dtype=dtype, tol=tol)
        th.join()
        mixed = srv.wait(tt, 120.0)
        rest = {i: srv.wait(t, 300.0) for i, t in tickets}
        st = srv.stats()
    assert mixed["status"] == P.LBM_OK
    assert mixed["iters"] == alone["iters"]
    # the same kernel advances each resident problem independently: identical
    assert np.array_equal(mixed["fields"], alone["fields"])
    assert rel_per_field(mixed["fields"], exact_fields(target)) < tol_fix
    assert st["peak_running"] > 1                     # requests overlapped on the device
    assert st["completed"] == len(others) + 1
    for i, r in rest.items():
        assert r["status"] == P.LBM_OK
        tf = 2e-5 if i % 2 else 2e-3
        assert rel_per_field(r["fields"], exact_fields(others[i])) < tf


def test_small_late_requests_finish_before_large_early_ones():
    """Continuous batching, not a FIFO queue: a small request submitted after
    a large one completes first."""
    big = problem(512, 512, 0.3, seed=7)
    small = problem(32, 32, 0.3, seed=8)
    with P.Server(4 * GIB, check_every=100) as srv:
        tb = srv.submit(*big[:6], tol=1e-8)
        time.sleep(0.05)
        ts = srv.submit(*small[:6], tol=1e-8)
        rs = srv.wait(ts, 60.0, fields=False)
        assert rs["status"] == P.LBM_OK
        assert srv.poll(tb, fields=False) is None      # the large one is still running
        rb = srv.wait(tb, 600.0, fields=False)
        assert rb["status"] == P.LBM_OK


def test_budget_limits_residency_and_queue_drains():
    probs = [problem(128, 128, 0.2, seed=200 + i) for i in range(12)]
    # 128^2 FP32 needs ~1.3 MB of arena; 8 MiB total gives each arena 4 MiB
    with P.Server(8 << 20, check_every=100) as srv:
        ts = [srv.submit(*p[:6], tol=1e-7) for p in probs]
        rs = [srv.wait(t, 300.0, fields=False) for t in ts]
        st = srv.stats()
    assert all(r["status"] == P.LBM_OK for r in rs)
    assert 1 <= st["peak_running"] <= 3
    assert st["completed"] == 12 and st["p99_ms"] >= st["p50_ms"] > 0
    # admission waited on memory, and the resident problems never exceeded the budget
    assert st["memory_waits"] > 0
    assert 0 < st["peak_resident_bytes"] <= 8 << 20


def test_host_side_faults():
    with P.Server(64 << 20, check_every=100) as srv:
        nx = ny = 16
        g = np.zeros((ny, nx))
        with pytest.raises(P.LBMError):                 # malformed: mu <= 0
            srv.submit(nx, ny, 0.3, -1.0, g, g)
        bad = g.copy()
        bad[3, 3] = np.nan
        with pytest.raises(P.LBMError):                 # non-finite force
            srv.submit(nx, ny, 0.3, 0.4, bad, g)
        huge = np.zeros((4096, 4096))
        with pytest.raises(P.LBMError):                 # larger than the budget
            srv.submit(4096, 4096, 0.3, 0.4, huge, huge)
        with pytest.raises(P.LBMError):                 # unknown ticket
            srv.poll(123456)
        # cancel a running request and a queued one; the server keeps working
        p = problem(256, 256, 0.3, seed=1)
        t1 = srv.submit(*p[:6], tol=1e-12)
        time.sleep(0.1)
        srv.cancel(t1)
        t2 = srv.submit(*problem(24, 24, 0.3, seed=2)[:6], tol=1e-8)
        r2 = srv.wait(t2, 60.0)
        assert r2["status"] == P.LBM_OK
        # an unpolled result stays available (slow consumer)
        t3 = srv.submit(*problem(20, 20, 0.3, seed=3)[:6], tol=1e-8)
        time.sleep(0.5)
        r3 = srv.poll(t3, fields=False)
        assert r3 is not None and r3["status"] == P.LBM_OK
        assert srv.stats()["failed"] == P.LBM_OK


def test_iteration_cap_and_divergence_reported():
    lam_u, mu_u = W.lame_2d(0.082, -0.4)
    pw = W.random_force(32, 32, 4, 3, seed=9)
    gx, gy = W.random_force_grid(pw)
    with P.Server(256 << 20, check_every=100) as srv:
        td = srv.submit(32, 32, lam_u, mu_u, gx, gy, tol=1e-12, max_iters=400_000)
        tc = srv.submit(*problem(64, 64, 0.3, seed=5)[:6], tol=1e-14, max_iters=250)
        rc = srv.wait(tc, 60.0, fields=False)
        rd = srv.wait(td, 300.0, fields=False)
    assert rc["status"] == P.LBM_ERR_NOT_CONVERGED and rc["iters"] == 300
    assert rd["status"] == P.LBM_ERR_DIVERGED
