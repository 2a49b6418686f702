"""Two pseudo-time steps per launch.  FP32 storage: the fused launch runs the
same per-node arithmetic as two single-step launches, so the state must agree
bit for bit with one step per launch, on ragged tiles, with general rates,
across residual-check windows, and through lbm_solve.  FP16-shifted storage:
the intermediate state stays in FP32, so the result must agree with one step
per launch, and with the oracle, within the FP16S storage tolerance (2e-3)."""
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


def _pair(nx, ny, seed=1, **kw):
    lam, mu = W.lame_2d(1.0, 0.3)
    pw = W.random_force(nx, ny, 8, 4, seed=seed)
    gx, gy = W.random_force_grid(pw)
    a = Lattice(nx, ny, lam, mu, "f32", **kw)
    b = Lattice(nx, ny, lam, mu, "f32", **kw)
    for lat in (a, b):
        lat.set_force(gx, gy)
    a.steps_per_launch = 1
    b.steps_per_launch = 2
    return a, b, gx, gy, lam, mu


# (64, 24) is the smallest lattice with two steps per launch; the others leave
# ragged tiles in x and/or y (tile 62 x 22 nodes).
@pytest.mark.parametrize("nx,ny", [(64, 24), (130, 70), (200, 97), (64, 300), (517, 33)])
@pytest.mark.parametrize("steps", [1, 2, 7])
def test_two_step_launch_is_bit_identical(nx, ny, steps):
    a, b, *_ = _pair(nx, ny)
    with a, b:
        a.iterate(steps)
        b.iterate(steps)
        assert a.step == b.step == steps
        fa, fb = a.populations(), b.populations()
        assert np.array_equal(fa, fb), float(np.max(np.abs(fa - fb)))


@pytest.mark.parametrize("kw", [dict(tau12=0.9, tau22=0.3), dict(theta=0.25)])
def test_two_step_general_rates_bit_identical(kw):
    a, b, *_ = _pair(150, 61, seed=2, **kw)
    with a, b:
        a.iterate(9)
        b.iterate(9)
        assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("check_every", [2, 7, 10])
def test_two_step_checked_windows(check_every):
    """Residual checks fall on the same steps and see the same maxima; the
    sums are reduced in another order (relative 1e-6)."""
    a, b, *_ = _pair(128, 96, seed=3)
    with a, b:
        ra = a.iterate_checked(41, check_every)
        rb = b.iterate_checked(41, check_every)
        assert np.array_equal(a.populations(), b.populations())
        assert ra[0] == rb[0] and ra[2] == rb[2] and ra[4] == rb[4]
        assert abs(ra[1] - rb[1]) <= 1e-6 * abs(ra[1]) and abs(ra[3] - rb[3]) <= 1e-6 * ra[3]


def test_two_step_solve_matches_single_step():
    a, b, *_ = _pair(96, 64, seed=4)
    with a, b:
        sa = a.solve(1e-6, 200000, 100)
        sb = b.solve(1e-6, 200000, 100)
        assert sa == sb, (sa, sb)
        assert np.array_equal(a.fields(), b.fields())


def test_two_step_matches_oracle():
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    nx, ny = 140, 71
    pw = W.random_force(nx, ny, 6, 4, seed=5)
    gx, gy = W.random_force_grid(pw)
    ref = oracle.run(oracle.zero_state(nx, ny), gx, gy, rates, 6)
    with Lattice(nx, ny, lam, mu, "f32") as lat:
        lat.steps_per_launch = 2
        lat.set_force(gx, gy)
        lat.iterate(6)
        got, want = lat.fields(), oracle.fields(ref, gx, gy, rates)
        err = max(float(np.max(np.abs(got[i] - want[i]))) / float(np.max(np.abs(want[i])))
                  for i in range(5))
        assert err < 2e-6, err


def test_steps_per_launch_availability():
    """Default for FP32 and FP16S: four steps from 256 x 8 on (wavefront
    schedule), else three from 64 x 16; any FP32/FP16S lattice may
    choose one to four; FP64 always one."""
    lam, mu = W.lame_2d(1.0, 0.3)
    for nx, ny, dt, want in ((64, 16, "f32", 3), (63, 32, "f32", 1), (64, 15, "f32", 1), (255, 64, "f32", 3),
                             (256, 8, "f32", 4), (256, 7, "f16s", 1), (300, 20, "f16s", 4),
                             (256, 256, "f64", 1), (256, 256, "f16s", 4), (63, 64, "f16s", 1)):
        with Lattice(nx, ny, lam, mu, dt) as lat:
            assert lat.steps_per_launch == want, (nx, ny, dt)
            lat.steps_per_launch = 1
            if dt == "f64":
                for k in (2, 3, 4):
                    with pytest.raises(P.LBMError):
                        lat.steps_per_launch = k
            else:
                for k in (2, 3, 4):
                    lat.steps_per_launch = k
                    assert lat.steps_per_launch == k
            for k in (0, 5):
                with pytest.raises(P.LBMError):
                    lat.steps_per_launch = k


# Lattices smaller than the 64 x 24 slot array appear in it more than once
# (periodic images); the result must still equal single steps bit for bit.
@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 3), (5, 5), (33, 17), (63, 23), (7, 130), (130, 7)])
def test_two_step_small_lattice_is_bit_identical(nx, ny):
    lam, mu = W.lame_2d(1.0, 0.3)
    pw = W.random_force(nx, ny, 4, 3, seed=9)
    gx, gy = W.random_force_grid(pw)
    out = []
    for spl in (1, 2):
        with Lattice(nx, ny, lam, mu, "f32") as lat:
            lat.steps_per_launch = spl
            lat.set_force(gx, gy)
            r = lat.iterate_checked(9, 3)
            out.append((lat.populations(), r))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1][0] == out[1][1][0]


def _rel(a, b):
    return max(float(np.max(np.abs(a[i] - b[i]))) / float(np.max(np.abs(b[i]))) for i in range(a.shape[0]))


@pytest.mark.parametrize("nx,ny", [(64, 24), (130, 70), (517, 33)])
def test_two_step_f16s_matches_single_step_and_oracle(nx, ny):
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    pw = W.random_force(nx, ny, 8, 4, seed=7)
    gx, gy = W.random_force_grid(pw)
    steps = 40
    ref = oracle.fields(oracle.run(oracle.zero_state(nx, ny), gx, gy, rates, steps), gx, gy, rates)
    out = {}
    for spl in (1, 2):
        with Lattice(nx, ny, lam, mu, "f16s") as lat:
            lat.steps_per_launch = spl
            lat.set_force(gx, gy)
            lat.iterate_checked(steps, 10)
            out[spl] = lat.fields()
    e1, e2, d12 = _rel(out[1], ref), _rel(out[2], ref), _rel(out[2], out[1])
    print("f16s one step/launch %.2e, two %.2e, between %.2e" % (e1, e2, d12))
    assert e1 < 2e-3 and e2 < 2e-3 and d12 < 2e-3


def test_two_step_f16s_conserves_mean_displacement():
    """The carriers keep the first moments of the stored state exactly, with
    or without the unrounded intermediate step."""
    lam, mu = W.lame_2d(1.0, 0.3)
    nx, ny = 128, 96
    pw = W.random_force(nx, ny, 8, 4, seed=8)
    gx, gy = W.random_force_grid(pw)
    with Lattice(nx, ny, lam, mu, "f16s") as lat:
        assert lat.steps_per_launch == 3
        lat.set_force(gx, gy)
        lat.iterate(2000)
        u = lat.displacement()
        scale = float(np.max(np.abs(u)))
        assert abs(float(np.mean(u[0]))) < 1e-4 * scale and abs(float(np.mean(u[1]))) < 1e-4 * scale


# Three steps per launch on the tile schedule (the wavefront schedule is
# switched off; its tests are in test_gpu_wavefront.py): tile 60 x 12 nodes,
# slot arrays 64 x 16.
@pytest.mark.parametrize("nx,ny", [(64, 16), (130, 70), (517, 33), (64, 300), (1, 1), (5, 5), (63, 15), (7, 130)])
@pytest.mark.parametrize("steps", [1, 2, 3, 7, 11])
def test_three_step_launch_is_bit_identical(nx, ny, steps):
    lam, mu = W.lame_2d(1.0, 0.3)
    pw = W.random_force(nx, ny, 8, 4, seed=31)
    gx, gy = W.random_force_grid(pw)
    out = []
    for spl in (1, 3):
        with Lattice(nx, ny, lam, mu, "f32") as lat:
            lat.steps_per_launch = spl
            lat.wavefront = 0
            lat.set_force(gx, gy)
            lat.iterate(steps)
            assert lat.step == steps
            out.append(lat.populations())
    assert np.array_equal(out[0], out[1]), float(np.max(np.abs(out[0] - out[1])))


@pytest.mark.parametrize("check_every", [2, 3, 7, 10])
def test_three_step_checked_windows_and_solve(check_every):
    lam, mu = W.lame_2d(1.0, 0.3)
    nx, ny = 128, 96
    pw = W.random_force(nx, ny, 8, 4, seed=32)
    gx, gy = W.random_force_grid(pw)
    res = []
    for spl in (1, 3):
        with Lattice(nx, ny, lam, mu, "f32", tau12=0.9, tau22=0.3) as lat:
            lat.steps_per_launch = spl
            lat.wavefront = 0
            lat.set_force(gx, gy)
            r = lat.iterate_checked(41, check_every)
            s = lat.solve(1e-6, 200000, 100)
            res.append((lat.populations(), r, s))
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1][0] == res[1][1][0] and res[0][1][2] == res[1][1][2]
    assert res[0][2] == res[1][2]


@pytest.mark.parametrize("nx,ny", [(64, 16), (130, 70)])
def test_three_step_f16s_matches_single_step_and_oracle(nx, ny):
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    pw = W.random_force(nx, ny, 8, 4, seed=33)
    gx, gy = W.random_force_grid(pw)
    steps = 42
    ref = oracle.fields(oracle.run(oracle.zero_state(nx, ny), gx, gy, rates, steps), gx, gy, rates)
    out = {}
    for spl in (1, 3):
        with Lattice(nx, ny, lam, mu, "f16s") as lat:
            lat.steps_per_launch = spl
            lat.wavefront = 0
            lat.set_force(gx, gy)
            lat.iterate_checked(steps, 7)
            out[spl] = lat.fields()
    e1, e3, d = _rel(out[1], ref), _rel(out[3], ref), _rel(out[3], out[1])
    print("f16s one step/launch %.2e, three %.2e, between %.2e" % (e1, e3, d))
    assert e1 < 2e-3 and e3 < 2e-3 and d < 2e-3
