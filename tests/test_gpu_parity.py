"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
  * FP64 storage: 1e-12 relative per step, 1e-10 relative at steady state
    (agreement with the oracle run for the same number of steps, and with the
    exact discrete fixed point when solved to a tight residual).
  * FP32 / FP16-shifted storage: the steady-state error against the FP64
    fixed point, relative to the field's maximum, must stay below the bound
    derived from the storage precision (FP32: 2e-5; FP16S: 2e-3 for
    displacement and stress); the measured errors are printed.
"""
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
from paper_2208_14870_gb300 import Lattice  # noqa: E402


def rel(a, b):
    s = max(float(np.max(np.abs(b))), 1e-300)
    return float(np.max(np.abs(a - b))) / s


def rel_per_field(a, b):
    return max(rel(a[i], b[i]) for i in range(a.shape[0]))


SIZES = [(1, 1), (2, 3), (3, 5), (4, 4), (5, 1), (1, 7), (33, 17), (130, 7), (64, 64),
         (127, 129), (257, 40)]


@pytest.mark.parametrize("nx,ny", SIZES)
def test_f64_single_step_matches_oracle(nx, ny):
    lam, mu = W.lame_2d(0.9, 0.25)
    rates = oracle.relaxation_rates(lam, mu)
    f = W.random_populations(8, nx, ny, seed=nx * 1000 + ny)
    gx = W.random_field(nx, ny, seed=1 + nx)
    gy = W.random_field(nx, ny, seed=2 + ny)
    with Lattice(nx, ny, lam, mu, "f64") as lat:
        lat.set_force(gx, gy)
        lat.set_populations(f)
        assert np.array_equal(lat.populations(), f)      # import/export is exact in FP64
        lat.iterate(1)
        got = lat.populations()
        ref = oracle.run(f, gx, gy, rates, 1)
        assert rel(got, ref) < 1e-12
        lat.iterate(4)
        ref = oracle.run(ref, gx, gy, rates, 4)
        assert rel(lat.populations(), ref) < 1e-12
        assert rel_per_field(lat.fields(), oracle.fields(ref, gx, gy, rates)) < 1e-12


def test_f64_general_rates_single_step():
    lam, mu = W.lame_2d(0.7, 0.25)
    t12, t22 = 0.9, 0.3
    rates = oracle.relaxation_rates(lam, mu, tau12=t12, tau22=t22)
    nx, ny = 37, 19
    f = W.random_populations(8, nx, ny, seed=5)
    gx = W.random_field(nx, ny, seed=6)
    gy = W.random_field(nx, ny, seed=7)
    with Lattice(nx, ny, lam, mu, "f64", tau12=t12, tau22=t22) as lat:
        r = lat.rates
        assert abs(r["w12"] - rates[3]) < 1e-15 and abs(r["w22"] - rates[5]) < 1e-15
        lat.set_force(gx, gy)
        lat.set_populations(f)
        lat.iterate(3)
        assert rel(lat.populations(), oracle.run(f, gx, gy, rates, 3)) < 1e-12


def test_theta_option_single_step():
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu, theta=0.25)
    nx, ny = 20, 12
    f = W.random_populations(8, nx, ny, seed=15)
    gx = W.random_field(nx, ny, seed=16)
    gy = W.random_field(nx, ny, seed=17)
    with Lattice(nx, ny, lam, mu, "f64", theta=0.25) as lat:
        lat.set_force(gx, gy)
        lat.set_populations(f)
        lat.iterate(2)
        assert rel(lat.populations(), oracle.run(f, gx, gy, rates, 2)) < 1e-12


@pytest.mark.parametrize("dtype,tol", [("f32", 2e-6), ("f16s", 2e-3)])
def test_low_precision_single_step(dtype, tol):
    """One step from a state the storage represents exactly enough: zero state
    with a random force, 3 steps."""
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    nx, ny = 150, 37
    pw = W.random_force(nx, ny, 6, 4, seed=3)
    gx, gy = W.random_force_grid(pw)
    ref = oracle.run(oracle.zero_state(nx, ny), gx, gy, rates, 3)
    with Lattice(nx, ny, lam, mu, dtype) as lat:
        lat.set_force(gx, gy)
        lat.iterate(3)
        assert rel_per_field(lat.fields(), oracle.fields(ref, gx, gy, rates)) < tol


def test_f64_plain_config_steady_state():
    """64 x 64, FP64, E = 1, nu = 0.3, manufactured sinusoidal force, residual
    1e-10: the GPU agrees with the oracle run for the same number of steps
    (1e-10), and, solved further to 1e-14, with the exact fixed point."""
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    man = W.sinusoid(64, 1, lam, mu)
    gx, gy = man.force()
    with Lattice(64, 64, lam, mu, "f64") as lat:
        lat.set_force(gx, gy)
        st, iters, r = lat.solve(1e-10, 10_000_000, 100)
        assert st == P.LBM_OK and r < 1e-10
        got = lat.fields()
        ref = oracle.fields(oracle.run(oracle.zero_state(64, 64), gx, gy, rates, iters), gx, gy, rates)
        assert rel_per_field(got, ref) < 1e-10
        st, more, r = lat.solve(1e-14, 10_000_000, 100)
        assert st == P.LBM_OK
        exact = oracle.fields(F.steady_state_grid(gx, gy, rates), gx, gy, rates)
        assert rel_per_field(lat.fields(), exact) < 1e-10
        # and the fixed point is second-order close to the PDE solution
        assert rel(lat.fields()[:2], man.exact()[:2]) < 5e-3


@pytest.mark.parametrize("dtype,tol_u,tol_s", [("f32", 2e-5, 2e-5), ("f16s", 2e-3, 2e-3)])
@pytest.mark.parametrize("n,k,nu", [(64, 1, 0.3), (128, 4, 0.45), (96, 1, 0.0)])
def test_low_precision_steady_state_error(dtype, tol_u, tol_s, n, k, nu):
    lam, mu = W.lame_2d(1.0, nu)
    rates = oracle.relaxation_rates(lam, mu)
    man = W.sinusoid(n, k, lam, mu)
    gx, gy = man.force()
    exact = oracle.fields(F.steady_state_grid(gx, gy, rates), gx, gy, rates)
    with Lattice(n, n, lam, mu, dtype) as lat:
        lat.set_force(gx, gy)
        st, iters, r = lat.solve(1e-9 if dtype == "f32" else 1e-7, 5_000_000, 500)
        assert st == P.LBM_OK, (st, iters, r)
        got = lat.fields()
        eu = rel_per_field(got[:2], exact[:2])
        es = rel_per_field(got[2:], exact[2:])
        print("%s n=%d k=%d nu=%.2f steps=%d: rel err u %.2e sigma %.2e" % (dtype, n, k, nu, iters, eu, es))
        assert eu < tol_u and es < tol_s


def test_rectangular_random_force_steady_state_f64():
    lam, mu = W.lame_2d(1.0, 0.2)
    rates = oracle.relaxation_rates(lam, mu)
    nx, ny = 72, 40
    pw = W.random_force(nx, ny, 8, 4, seed=11)
    gx, gy = W.random_force_grid(pw)
    ks, fh, flh = F.steady_state_modes(nx, ny, pw.modes(), rates)
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    exact = np.stack([F.evaluate_modes(ks, flh[:, c], X, Y) for c in range(5)])
    with Lattice(nx, ny, lam, mu, "f64") as lat:
        lat.set_force(gx, gy)
        st, iters, r = lat.solve(1e-14, 10_000_000, 200)
        assert st == P.LBM_OK
        assert rel_per_field(lat.fields(), exact) < 1e-10


def test_residual_definition_matches_oracle():
    """Checks every k = 10 steps well before steady state (slow k = 1 mode)."""
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    nx, ny = 64, 48
    man = W.sinusoid(nx, 1, lam, mu, ny=ny)
    gx, gy = man.force()
    with Lattice(nx, ny, lam, mu, "f64") as lat:
        lat.set_force(gx, gy)
        # checks fused into steps 10, 20, 30 measure u at their input times
        # 9, 19, 29; the last residual compares u^29 with u^19
        out = lat.iterate_checked(30, 10)
    f20 = oracle.run(oracle.zero_state(nx, ny), gx, gy, rates, 19)
    f30 = oracle.run(f20, gx, gy, rates, 10)
    u20 = oracle.fields(f20, gx, gy, rates)[:2]
    u30 = oracle.fields(f30, gx, gy, rates)[:2]
    r_inf, r_2 = oracle.residual(u30, u20, 10)
    assert r_inf > 1e-4
    assert abs(out[0] - r_inf) < 1e-12 * r_inf
    assert abs(out[1] - r_2) < 1e-12 * r_2
    assert abs(out[2] - np.max(np.abs(u30))) < 1e-14 * np.max(np.abs(u30))
    assert out[4] == 0.0


def test_divergence_is_reported_at_unstable_point():
    """nu = -0.4, E~ = 0.082 lies outside the stable region (Sec. 6.3.5)."""
    lam, mu = W.lame_2d(0.082, -0.4)
    nx = ny = 32
    f = W.random_populations(8, nx, ny, seed=9, scale=1e-3)
    z = np.zeros((ny, nx))
    with Lattice(nx, ny, lam, mu, "f32") as lat:
        lat.set_force(z, z)
        lat.set_populations(f)
        st, iters, r = lat.solve(1e-8, 400_000, 1000)
        assert st == P.LBM_ERR_DIVERGED
        assert iters < 400_000


def test_zero_force_stays_zero_and_solve_converges_immediately():
    lam, mu = W.lame_2d(1.0, 0.3)
    z = np.zeros((9, 11))
    for dtype in ("f64", "f32", "f16s"):
        with Lattice(11, 9, lam, mu, dtype) as lat:
            lat.set_force(z, z)
            st, iters, r = lat.solve(1e-4, 10_000, 10)
            # first check takes the snapshot, the second sees r = 0
            assert st == P.LBM_OK and r == 0.0 and iters == 20
            assert not np.any(lat.fields())
            # a tolerance below the storage's rounding floor for 10-step windows
            # is checked over longer windows (a multiple of 10 steps)
            lat.reset()
            st, iters, r = lat.solve(1e-9, 100_000, 10)
            assert st == P.LBM_OK and r == 0.0 and iters % 10 == 0 and iters >= 20


def test_device_fields_match_host_fields_and_stream_interop():
    lam, mu = W.lame_2d(1.0, 0.3)
    nx, ny = 200, 60
    pw = W.random_force(nx, ny, 4, 3, seed=8)
    gx, gy = W.random_force_grid(pw)
    s = torch.cuda.Stream()
    with Lattice(nx, ny, lam, mu, "f32") as lat:
        lat.set_stream(s.cuda_stream)
        lat.set_force(torch.tensor(gx, device="cuda"), torch.tensor(gy, device="cuda"))
        lat.iterate(50)
        out = torch.empty(5 * nx * ny, dtype=torch.float64, device="cuda")
        lat.fields_device(out)
        s.synchronize()
        host = lat.fields()
        assert np.array_equal(out.cpu().numpy().reshape(5, ny, nx), host)


def test_reset_restores_zero_state():
    lam, mu = W.lame_2d(1.0, 0.3)
    nx, ny = 50, 30
    gx = W.random_field(nx, ny, seed=1, zero_mean=True)
    gy = W.random_field(nx, ny, seed=2, zero_mean=True)
    for dtype in ("f64", "f32", "f16s"):
        with Lattice(nx, ny, lam, mu, dtype) as lat:
            lat.set_force(gx, gy)
            lat.iterate(7)
            a = lat.fields()
            lat.reset()
            assert lat.step == 0
            lat.iterate(7)
            assert np.array_equal(lat.fields(), a)


def test_f16s_force_rescale_keeps_state():
    """Changing the force magnitude rescales the stored FP16 deviations by a
    power of two: exact when the scale grows (force made smaller); when it
    shrinks, the smallest deviations lose bits as they move toward FP16's
    subnormal range."""
    lam, mu = W.lame_2d(1.0, 0.3)
    nx, ny = 64, 48
    pw = W.random_force(nx, ny, 4, 3, seed=21)
    gx, gy = W.random_force_grid(pw)
    with Lattice(nx, ny, lam, mu, "f16s") as lat:
        lat.set_force(gx, gy)
        lat.iterate(40)
        before = lat.populations()
        lat.set_force(gx / 1024.0, gy / 1024.0)
        assert np.array_equal(lat.populations(), before)
        lat.set_force(gx * 1024.0, gy * 1024.0)
        assert rel(lat.populations(), before) < 1e-4


@pytest.mark.parametrize("dtype", ["f32", "f16s"])
def test_full_size_sampled_parity(dtype):
    """16384 x 16384 (the throughput workload) in the benchmark's launch
    configuration: one plain four-step wavefront launch (k_wave, 128-row
    segments) and one four-step wavefront launch whose last level carries the
    residual check, as every residual window of the benchmark ends.  After 8
    steps from the zero state every node depends on the force within 8 nodes,
    so sampled nodes are checked one by one against the oracle run on a
    small periodic window (19 x 19) around each sample."""
    n = 16384
    steps = 8
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    pw = W.random_force(n, n, 16, 8, seed=0x16384)
    gx, gy = W.random_force_grid(pw)
    with Lattice(n, n, lam, mu, dtype) as lat:
        assert lat.steps_per_launch == 4 and lat.wavefront == -1
        lat.set_force(gx, gy)
        lat.iterate(4)                  # one plain four-step wavefront launch
        lat.iterate_checked(4, 4)       # and one checked four-step wavefront launch
        out = torch.empty(5 * n * n, dtype=torch.float64, device="cuda")
        lat.fields_device(out)
        got = out.view(5, n, n)
        rng = np.random.Generator(np.random.PCG64(5))
        pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0)] + [
            tuple(int(v) for v in rng.integers(0, n, 2)) for _ in range(60)]
        w = 2 * steps + 3
        h = w // 2
        worst = 0.0
        for (x0, y0) in pts:
            ys = [(y0 + d) % n for d in range(-h, h + 1)]
            xs = [(x0 + d) % n for d in range(-h, h + 1)]
            wx = np.ascontiguousarray(gx[np.ix_(ys, xs)])
            wy = np.ascontiguousarray(gy[np.ix_(ys, xs)])
            ref = oracle.fields(oracle.run(oracle.zero_state(w, w), wx, wy, rates, steps), wx, wy, rates)
            g = got[:, y0, x0].cpu().numpy()
            scale = np.max(np.abs(ref[:, h, h])) + 1e-300
            worst = max(worst, float(np.max(np.abs(g - ref[:, h, h]))) / scale)
        assert worst < (2e-6 if dtype == "f32" else 2e-3), worst
        del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5), ("f16s", 1e-4)])
def test_mean_displacement_is_conserved(dtype, tol):
    """With a zero-mean force the mean of u is conserved (Sec. 6.2; exact
    first-moment balance).  The FP16-shifted store keeps the first moments of
    the stored state exact, so rounding cannot drift the mean either."""
    lam, mu = W.lame_2d(1.0, 0.3)
    nx, ny = 40, 33
    pw = W.random_force(nx, ny, 4, 3, seed=123)
    gx, gy = W.random_force_grid(pw)
    with Lattice(nx, ny, lam, mu, dtype) as lat:
        lat.set_force(gx, gy)
        lat.iterate(20000)
        u = lat.displacement()
    scale = float(np.max(np.abs(u)))
    assert abs(float(u[0].mean())) < tol * scale and abs(float(u[1].mean())) < tol * scale


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 2e-5)])
def test_force_correction_matches_oracle(dtype, tol):
    """lbm_set_force_corrected applies the higher-order force correction on
    the device; the steady state equals the exact fixed point of the oracle's
    corrected force (same central differences)."""
    lam, mu = W.lame_2d(0.3, 0.25)
    rates = oracle.relaxation_rates(lam, mu)
    nx, ny = 48, 40
    pw = W.random_force(nx, ny, 4, 3, seed=31)
    gx, gy = W.random_force_grid(pw)
    D = np.array([0.152, -0.016, -0.0199])
    gxc, gyc = oracle.corrected_force_fd(gx, gy, D)
    exact = oracle.fields(F.steady_state_grid(gxc, gyc, rates), gxc, gyc, rates)
    with Lattice(nx, ny, lam, mu, dtype) as lat:
        lat.set_force_corrected(gx, gy, D)
        st, iters, r = lat.solve(1e-14 if dtype == "f64" else 2e-9, 10_000_000, 200)
        assert st == P.LBM_OK
        assert rel(lat.fields()[:2], exact[:2]) < tol


def test_host_field_getters_follow_every_state_change():
    """lbm_get_displacement and lbm_get_stress share one field recovery per
    state; after a step, a new force, a reset, a population read-back or a
    population load they must show the new state (each checked against the
    device-side recovery, which never uses the shared one)."""
    lam, mu = W.lame_2d(1.0, 0.3)
    nx, ny = 96, 40
    pw = W.random_force(nx, ny, 6, 4, seed=21)
    gx, gy = W.random_force_grid(pw)
    with Lattice(nx, ny, lam, mu, "f32") as lat:
        dev = torch.empty(5 * nx * ny, dtype=torch.float64, device="cuda")

        def check():
            host = np.concatenate([lat.displacement(), lat.stress()])
            want = lat.fields_device(dev).view(5, ny, nx).cpu().numpy()
            assert np.array_equal(host, want)
            return host

        lat.set_force(gx, gy)
        lat.iterate(7)
        a = check()
        lat.iterate(3)
        b = check()
        assert not np.array_equal(a, b)
        lat.set_force(0.5 * gx, 0.5 * gy)          # u = m10 + g/2 changes with g
        c = check()
        assert not np.array_equal(b, c)
        f = lat.populations()
        check()
        lat.reset()
        z = check()                               # zero state: u = g/2, sigma = 0
        assert np.allclose(z[0], 0.25 * gx) and np.max(np.abs(z[2:])) == 0.0
        lat.set_populations(f)
        assert np.array_equal(check(), c)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
def test_pinned_and_pageable_host_buffers_agree(dtype):
    """lbm_set_force reads pinned host arrays with the conversion kernel over
    the host link, and the field getters write pinned host arrays from the
    recovery kernel; pageable arrays go through device staging copies.  Both
    routes give the same bits, and a non-finite entry is rejected on both."""
    lam, mu = W.lame_2d(1.0, 0.3)
    nx, ny = 300, 70
    pw = W.random_force(nx, ny, 6, 4, seed=99)
    gx, gy = W.random_force_grid(pw)
    pgx = torch.from_numpy(gx.copy()).pin_memory()
    pgy = torch.from_numpy(gy.copy()).pin_memory()
    out = []
    for pinned in (False, True):
        with Lattice(nx, ny, lam, mu, dtype) as lat:
            if pinned:
                P.lbm_set_force(lat.ctx, pgx.data_ptr(), pgy.data_ptr())
            else:
                P.lbm_set_force(lat.ctx, gx.ctypes.data, gy.ctypes.data)
            lat.iterate(37)
            if pinned:
                f = [torch.empty(nx * ny, dtype=torch.float64).pin_memory() for _ in range(5)]
                P.lbm_get_displacement(lat.ctx, f[0].data_ptr(), f[1].data_ptr())
                P.lbm_get_stress(lat.ctx, f[2].data_ptr(), f[3].data_ptr(), f[4].data_ptr())
                out.append(np.stack([t.numpy().reshape(ny, nx) for t in f]))
            else:
                out.append(np.concatenate([lat.displacement(), lat.stress()]))
            bad = pgx.clone().pin_memory()
            bad[5] = float("nan")
            with pytest.raises(P.LBMError):
                P.lbm_set_force(lat.ctx, bad.data_ptr(), pgy.data_ptr())
    assert np.array_equal(out[0], out[1])


def _pinned_solve(nx, ny, lam, mu, dtype, pgx, pgy, steps, mode, stream=None):
    """Force from pinned arrays, `steps` steps, the five fields into pinned
    arrays, with host transfer `mode` (optionally on its own stream)."""
    with Lattice(nx, ny, lam, mu, dtype) as lat:
        if stream is not None:
            lat.set_stream(stream.cuda_stream)
        lat.host_transfer = mode
        assert lat.host_transfer == mode
        P.lbm_set_force(lat.ctx, pgx.data_ptr(), pgy.data_ptr())
        lat.iterate(steps)
        f = [torch.empty(nx * ny, dtype=torch.float64).pin_memory() for _ in range(5)]
        P.lbm_get_displacement(lat.ctx, f[0].data_ptr(), f[1].data_ptr())
        P.lbm_get_stress(lat.ctx, f[2].data_ptr(), f[3].data_ptr(), f[4].data_ptr())
        return np.stack([t.numpy().reshape(ny, nx) for t in f])


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
def test_host_copy_mode_agrees_with_direct(dtype):
    """LBM_HOST_COPY moves pinned host arrays by copies through device staging
    instead of kernels that read and write them over the host link: the same
    bits; an unknown mode is rejected."""
    lam, mu = W.lame_2d(1.0, 0.3)
    nx, ny = 300, 70
    gx, gy = W.random_force_grid(W.random_force(nx, ny, 6, 4, seed=98))
    pgx = torch.from_numpy(gx.copy()).pin_memory()
    pgy = torch.from_numpy(gy.copy()).pin_memory()
    a = _pinned_solve(nx, ny, lam, mu, dtype, pgx, pgy, 41, P.LBM_HOST_DIRECT)
    b = _pinned_solve(nx, ny, lam, mu, dtype, pgx, pgy, 41, P.LBM_HOST_COPY)
    assert np.array_equal(a, b)
    with Lattice(8, 8, lam, mu, dtype) as lat:
        with pytest.raises(P.LBMError):
            lat.host_transfer = 2


def test_two_lattices_on_two_streams_from_two_threads():
    """Two lattices on their own streams, driven from two host threads with
    copy-engine transfers (the pipelined end-to-end form of the benchmark):
    each gives the bits it gives alone."""
    import threading
    lam, mu = W.lame_2d(1.0, 0.3)
    nx, ny = 512, 260
    cases = []
    for seed in (11, 12):
        gx, gy = W.random_force_grid(W.random_force(nx, ny, 8, 4, seed=seed))
        cases.append((torch.from_numpy(gx.copy()).pin_memory(), torch.from_numpy(gy.copy()).pin_memory()))
    alone = [_pinned_solve(nx, ny, lam, mu, "f32", gx, gy, 64, P.LBM_HOST_COPY) for gx, gy in cases]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    got = [None, None]
    errors = []

    def run(k):
        try:
            for _ in range(3):
                got[k] = _pinned_solve(nx, ny, lam, mu, "f32", *cases[k], 64, P.LBM_HOST_COPY, streams[k])
        except Exception as e:  # pragma: no cover - reported below
            errors.append(e)

    threads = [threading.Thread(target=run, args=(k,)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for k in range(2):
        assert np.array_equal(got[k], alone[k])
