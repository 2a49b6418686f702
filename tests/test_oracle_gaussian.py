"""The Gaussian-hill workload of Sec. 6.3.5: second-order convergence of the
exact discrete steady state to the manufactured field, and the stability pair
at nu = -0.4 (E~ = 0.082 diverges under time stepping, a stable E~ converges)."""
import numpy as np

import oracle
import oracle.fourier as F
import workloads as W


def test_gaussian_hill_second_order():
    lam, mu = W.lame_2d(1.0, 0.3)
    rates = oracle.relaxation_rates(lam, mu)
    eu, es = [], []
    for n in (64, 128, 256):
        gx, gy, ex = W.gaussian_hill(n, lam, mu)
        fl = oracle.fields(F.steady_state_grid(gx, gy, rates), gx, gy, rates)
        eu.append(np.max(np.abs(fl[:2] - ex[:2])) / np.max(np.abs(ex[:2])))
        es.append(np.max(np.abs(fl[2:] - ex[2:])) / np.max(np.abs(ex[2:])))
    for e in (eu, es):
        r = np.array(e[:-1]) / np.array(e[1:])
        assert np.all(r > 3.5) and np.all(r < 4.5), r


def test_gaussian_hill_stability_pair():
    """Sec. 6.3.5: with the dense spectrum of the hill, nu = -0.4 and
    E~ = 0.082 (outside the stable region) blow up; E~ = 0.3 converges."""
    n = 32
    out = {}
    for E in (0.082, 0.3):
        lam, mu = W.lame_2d(E, -0.4)
        rates = oracle.relaxation_rates(lam, mu)
        gx, gy, ex = W.gaussian_hill(n, lam, mu)
        f = oracle.run(oracle.zero_state(n, n), gx, gy, rates, 6000)
        out[E] = np.max(np.abs(oracle.fields(f, gx, gy, rates)[:2])) / np.max(np.abs(ex[:2]))
    assert out[0.082] > 1e6
    assert 0.5 < out[0.3] < 2.0
