"""Wavefront schedule of three or four pseudo-time steps per launch
(lbm_set_wavefront).  FP32 storage: every launch runs the single step's
per-node arithmetic, so the state must agree bit for bit with one step per
launch -- on ragged strips (256 slot columns, 252 or 250 outputs) and ragged
segments, segments of one row, general rates, residual-check windows and
lbm_solve.  FP16-shifted storage: within the storage tolerance (2e-3) of one
step per launch and of the oracle."""
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


def _run(nx, ny, dtype, spl, wave, steps, seed, check_every=None, **kw):
    lam, mu = W.lame_2d(1.0, 0.3)
    pw = W.random_force(nx, ny, 8, 4, seed=seed)
    gx, gy = W.random_force_grid(pw)
    with Lattice(nx, ny, lam, mu, dtype, **kw) as lat:
        lat.steps_per_launch = spl
        lat.wavefront = wave
        lat.set_force(gx, gy)
        r = lat.iterate_checked(steps, check_every) if check_every else lat.iterate(steps)
        assert lat.step == steps
        return lat.populations(), r, lat.fields()


# (256, 8): one strip, the smallest lattice on the schedule; the others leave
# a ragged last strip and/or segment (268, 500: the last strip reaches past
# the lattice's x period by a few to 247 columns).
@pytest.mark.parametrize("nx,ny", [(256, 8), (256, 45), (293, 40), (509, 23), (763, 13), (1000, 77),
                                   (264, 8), (268, 9), (500, 16), (752, 33)])
@pytest.mark.parametrize("T", [3, 4])
@pytest.mark.parametrize("seg", [1, 7, 128, -1])
@pytest.mark.parametrize("steps", [None, 11])
def test_wavefront_is_bit_identical(nx, ny, T, seg, steps):
    steps = T if steps is None else steps
    a = _run(nx, ny, "f32", 1, 0, steps, 41)[0]
    b = _run(nx, ny, "f32", T, seg, steps, 41)[0]
    assert np.array_equal(a, b), float(np.max(np.abs(a - b)))


@pytest.mark.parametrize("kw", [dict(tau12=0.9, tau22=0.3), dict(theta=0.25)])
@pytest.mark.parametrize("T", [3, 4])
def test_wavefront_general_rates_bit_identical(kw, T):
    a = _run(300, 50, "f32", 1, 0, 13, 42, **kw)[0]
    b = _run(300, 50, "f32", T, 16, 13, 42, **kw)[0]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("check_every", [2, 3, 7, 10])
@pytest.mark.parametrize("T", [3, 4])
def test_wavefront_checked_windows_and_solve(check_every, T):
    lam, mu = W.lame_2d(1.0, 0.3)
    nx, ny = 300, 64
    pw = W.random_force(nx, ny, 8, 4, seed=43)
    gx, gy = W.random_force_grid(pw)
    res = []
    for spl, wave in ((1, 0), (T, 32)):
        with Lattice(nx, ny, lam, mu, "f32", tau12=0.9, tau22=0.3) as lat:
            lat.steps_per_launch = spl
            lat.wavefront = wave
            lat.set_force(gx, gy)
            r = lat.iterate_checked(41, check_every)
            s = lat.solve(1e-6, 200000, 100)
            res.append((lat.populations(), r, s))
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1][0] == res[1][1][0] and res[0][1][2] == res[1][1][2]
    assert res[0][2] == res[1][2]


def test_wavefront_large_lattice_bit_identical():
    """A lattice of many strips and segments at the default segment length."""
    a = _run(2048, 1100, "f32", 1, 0, 9, 44)[0]
    b = _run(2048, 1100, "f32", 4, 128, 9, 44)[0]
    assert np.array_equal(a, b)


def _rel(a, b):
    return max(float(np.max(np.abs(a[i] - b[i]))) / float(np.max(np.abs(b[i]))) for i in range(a.shape[0]))


@pytest.mark.parametrize("nx,ny", [(300, 70), (517, 33)])
@pytest.mark.parametrize("T", [3, 4])
def test_wavefront_f16s_matches_single_step_and_oracle(nx, ny, T):
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    pw = W.random_force(nx, ny, 8, 4, seed=45)
    gx, gy = W.random_force_grid(pw)
    steps = 42
    ref = oracle.fields(oracle.run(oracle.zero_state(nx, ny), gx, gy, rates, steps), gx, gy, rates)
    one = _run(nx, ny, "f16s", 1, 0, steps, 45, check_every=7)[2]
    wav = _run(nx, ny, "f16s", T, 16, steps, 45, check_every=7)[2]
    e1, ew, d = _rel(one, ref), _rel(wav, ref), _rel(wav, one)
    print("f16s one step/launch %.2e, wavefront x%d %.2e, between %.2e" % (e1, T, ew, d))
    assert e1 < 2e-3 and ew < 2e-3 and d < 2e-3


def test_wavefront_settings():
    """Default -1 (segments chosen per launch) for FP32/FP16S, 0 for FP64; four
    steps per launch run as three where the schedule is off or the lattice is
    narrower than a strip."""
    lam, mu = W.lame_2d(1.0, 0.3)
    for dt, want in (("f32", -1), ("f16s", -1), ("f64", 0)):
        with Lattice(256, 16, lam, mu, dt) as lat:
            assert lat.wavefront == want
            with pytest.raises(P.LBMError):
                lat.wavefront = -2
            if dt == "f64":
                for rows in (8, -1):
                    with pytest.raises(P.LBMError):
                        lat.wavefront = rows
            else:
                lat.wavefront = 0
                assert lat.wavefront == 0
                lat.steps_per_launch = 4
                assert lat.steps_per_launch == 4
    for nx, ny, wave in ((255, 40, 128), (300, 40, 0), (256, 7, 64), (600, 500, -1)):
        a = _run(nx, ny, "f32", 1, 0, 10, 46)[0]
        b = _run(nx, ny, "f32", 4, wave, 10, 46)[0]
        assert np.array_equal(a, b), (nx, ny, wave)
