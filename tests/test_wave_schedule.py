"""Host check of the wavefront schedule of k_wave (no GPU): the kernel's level
windows, its two-row lag between step levels, its four-row shared-memory
rings of six populations, the per-thread delay lines that carry populations 2
and 4 (the vertical movers, pulled from the thread's own column) across each
level boundary, and its register history of the force (level j reads the
entry 2(j - 1) rows back), replayed block by block in numpy on a toy per-node
update with the same pull streaming, must give exactly T single steps -- every
ring read finds the row it needs, every delay-line read the row it needs,
every slot index stays inside its ring row, every output node is written
once, and the periodic wrap of slot coordinates stays within one period.  The
constants (ring depth, warps per block) are read from the kernel header so
that the replay follows the compiled schedule."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT

C = [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
RING = [0, 2, 4, 5, 6, 7]          # populations held in the shared-memory rings


def _constants():
    src = open(os.path.join(ROOT, "paper_2208_14870_gb300", "csrc", "lbm_kernels.cuh")).read()
    depth = int(re.search(r"constexpr int kWvD = (\d+);", src).group(1))
    nw = int(re.search(r"#define LBM_WV_NW (\d+)", src).group(1))
    return depth, 32 * nw


def _toy(f, gx, gy):
    # any per-node map mixing all populations and the force, with exactly
    # rounded operations only (so the replay order cannot change the bits)
    s = f[0].copy()
    for q in range(1, 8):
        s = s + f[q]
    return np.stack([0.125 * f[p] * (p + 1) - 0.1 * s * f[(p + 3) % 8] + 0.01 * gx - 0.02 * gy * p
                     for p in range(8)])


def _single(state, gx, gy):
    f = np.empty_like(state)
    for p, (cx, cy) in enumerate(C):
        f[p] = np.roll(np.roll(state[p], cy, axis=0), cx, axis=1)   # f_p(x) = f*_p(x - c_p)
    return _toy(f, gx, gy)


def _wrap_slot(v, n):
    assert -n <= v < 2 * n        # one conditional add or subtract suffices
    return v + n if v < 0 else (v - n if v >= n else v)


def _wave(state, gx, gy, T, seg, W, D):
    ny, nx = gx.shape
    OX = W - 2 * (T - 1)
    nstrips = -(-nx // OX)
    nsegs = -(-ny // seg)
    out = np.full_like(state, np.nan)
    written = np.zeros((ny, nx), int)
    t = np.arange(W)
    for b in range(nstrips * nsegs):
        strip, y0 = b % nstrips, (b // nstrips) * seg
        rows = min(seg, ny - y0)
        xs = strip * OX - (T - 1) + t
        x = np.array([_wrap_slot(v, nx) for v in xs])
        store_ok = (t >= T - 1) & (t <= W - T) & (xs < nx)
        ring = np.full((T - 1, 8, D, W), np.nan)
        held = np.full((T - 1, D), -10 ** 9)          # lattice row held by each ring slot
        ybeg = y0 - (T - 1)
        hist = [None] * (2 * (T - 1) + 1)              # force rows held in registers
        nan_row = (None, np.full(W, np.nan))
        v2 = [[nan_row] * 3 for _ in range(T - 1)]      # (row, values): last three productions
        v4 = [nan_row] * (T - 1)                        # (row, values): last production
        n1 = rows + 2 * (T - 1)
        for i in range(rows + 3 * (T - 1)):
            writes = []                                # applied after the block barrier
            reads = set()                              # ring slots read in this iteration
            hist = [ybeg + i if i < rows + 2 * (T - 1) else None] + hist[:-1]
            for tau in range(T, 1, -1):
                if i < 3 * (tau - 1) or i > rows + 2 * T + tau - 4:
                    continue
                yl = ybeg + i - 2 * (tau - 1)
                assert hist[2 * (tau - 1)] == yl       # the register history holds this row's force
                act = store_ok if tau == T else (t >= tau - 1) & (t <= W - tau)
                for dy in (-1, 0, 1):
                    assert held[tau - 2][(yl + dy) % D] == yl + dy
                    reads.add((tau - 2, (yl + dy) % D))
                f = np.empty((8, int(act.sum())))
                for p in RING:
                    cx, cy = C[p]
                    cols = t[act] - cx
                    assert cols.min() >= 0 and cols.max() < W
                    f[p] = ring[tau - 2][p][(yl - cy) % D][cols]
                row, val = v2[tau - 2][2]              # population 2: c = (0, 1), from row yl - 1
                assert row == yl - 1
                f[1] = val[act]
                row, val = v4[tau - 2]                 # population 4: c = (0, -1), from row yl + 1
                assert row == yl + 1
                f[3] = val[act]
                assert not np.isnan(f).any()
                yw = _wrap_slot(yl, ny)
                g = _toy(f, gx[yw, x[act]], gy[yw, x[act]])
                if tau < T:
                    writes.append((tau - 1, yl, act, g))
                    # the delay lines shift as the producer runs (after this
                    # iteration's consumer of the same boundary has read them)
                    p2, p4 = np.full(W, np.nan), np.full(W, np.nan)
                    p2[act], p4[act] = g[1], g[3]
                    v2[tau - 1] = [(yl, p2)] + v2[tau - 1][:2]
                    v4[tau - 1] = (yl, p4)
                else:
                    assert 0 <= yl < ny and (xs[act] == x[act]).all()
                    out[:, yl, x[act]] = g
                    written[yl, x[act]] += 1
            if i < n1:
                y1 = ybeg + i
                y = _wrap_slot(y1, ny)
                f = np.empty((8, W))
                for p, (cx, cy) in enumerate(C):
                    f[p] = state[p][(y - cy) % ny][(x - cx) % nx]
                g = _toy(f, gx[y, x], gy[y, x])
                writes.append((0, y1, np.ones(W, bool), g))
                v2[0] = [(y1, g[1])] + v2[0][:2]
                v4[0] = (y1, g[3])
            # threads of one iteration are not ordered: no slot may be both
            # read and written between two barriers
            assert not reads & {(lv, yl % D) for lv, yl, _, _ in writes}
            for lv, yl, act, g in writes:
                ring[lv][:, yl % D, :] = np.nan
                held_vals = np.full((len(RING), W), np.nan)
                held_vals[:, act] = g[RING]
                ring[lv][RING, yl % D, :] = held_vals
                held[lv][yl % D] = yl
    assert (written == 1).all()
    return out


D, W_KERNEL = _constants()


@pytest.mark.parametrize("W", [32, W_KERNEL])
@pytest.mark.parametrize("T", [3, 4])
@pytest.mark.parametrize("dnx,ny,seg", [(0, 8, 100), (3, 8, 3), (0, 8, 8), (1, 9, 4), (-3, 23, 7),
                                          (37, 40, 16), (0, 31, 31), (5, 17, 1)])
def test_wavefront_schedule_equals_single_steps(W, T, dnx, ny, seg):
    nx = (2 * W if dnx < 0 else W) + dnx       # from one strip width up, ragged last strip
    if W == W_KERNEL and (ny > 24 or seg == 1):
        pytest.skip("the kernel-width replay covers the short cases")
    rng = np.random.default_rng(nx * 131 + ny * 7 + T + seg)
    state = rng.standard_normal((8, ny, nx))
    gx = rng.standard_normal((ny, nx))
    gy = rng.standard_normal((ny, nx))
    ref = state
    for _ in range(T):
        ref = _single(ref, gx, gy)
    got = _wave(state, gx, gy, T, seg, W, D)
    assert np.array_equal(got, ref)


def test_ring_depth_is_the_minimum():
    """Level j + 1 reads rows r - 3 .. r - 1 of level j while level j writes
    row r in the same iteration: with three ring rows the slot of row r - 3
    is read and written between the same two barriers."""
    assert D == 4
    rng = np.random.default_rng(5)
    nx, ny = 40, 12
    state = rng.standard_normal((8, ny, nx))
    g = rng.standard_normal((2, ny, nx))
    with pytest.raises(AssertionError):
        _wave(state, g[0], g[1], 3, 6, 32, 3)
