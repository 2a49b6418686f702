"""Host-side checks of bench.py's bookkeeping (no GPU): the launch count of a
residual-checked iteration, the comment-insensitive kernel-code hash that
keys the recorded DRAM traffic (a stale record reads as null in the bench
line), and the host description of the CPU baseline."""
import importlib.util
import os

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def simulate_launches(iters, check_every, spl, wave=False):
    """Launch sequence of lbm_iterate_checked from step 0, written out launch
    by launch as the library plans it: plain steps grouped into launches of spl
    steps (four only on the wavefront schedule, else three), leftovers in
    shorter launches, and a check step (index + 1 a multiple of check_every)
    as the last step of a four-step wavefront launch (where the schedule runs
    four steps per launch and the window has at least four steps), else of a
    launch of at most two steps."""
    big = 4 if spl >= 4 and wave else min(spl, 3)

    def plain(m):
        count = 0
        while m > 0:
            k = min(big, m)
            if big == 3 and m == 4:
                k = 2          # 4 = 2 + 2 instead of 3 + 1
            if big == 4 and m == 5:
                k = 3          # 5 = 3 + 2 instead of 4 + 1
            m -= k
            count += 1
        return count
    launches, step, left = 0, 0, iters
    while left > 0:
        to_check = check_every - step % check_every
        if to_check > left:
            launches += plain(left)
            break
        # the check rides on a four-step wavefront launch or a launch of at most two steps
        last = 4 if (spl >= 4 and wave and to_check >= 4) else min(spl, 2, to_check)
        launches += plain(to_check - last) + 1
        step += to_check
        left -= to_check
    return launches


@pytest.mark.parametrize("spl,wave", [(1, False), (2, False), (3, False), (3, True), (4, False), (4, True)])
def test_launch_count_matches_the_schedule(bench, spl, wave):
    for iters in (0, 1, 2, 5, 7, 9, 99, 100, 101, 1000, 1234):
        for ce in (1, 2, 3, 6, 7, 10, 11, 100):
            assert (bench.launches_per_iterate(iters, ce, spl, wave)
                    == simulate_launches(iters, ce, spl, wave)), (iters, ce)
    assert bench.launches_per_iterate(1000, 100, 2) == 500
    assert bench.launches_per_iterate(1000, 100, 1) == 1000
    assert bench.launches_per_iterate(1000, 100, 3) == 10 * (33 + 1)   # 98 = 32 x 3 + 2, then the check pair
    assert bench.launches_per_iterate(1000, 100, 4, True) == 10 * 25   # 96 = 24 x 4, then the checked four


def test_dominant_block(bench):
    # the first steps of a window that run as whole launches of the longest kind
    assert bench.dominant_block(100, 1) == (99, 1)
    assert bench.dominant_block(100, 2) == (98, 2)
    assert bench.dominant_block(100, 3) == (96, 3)
    assert bench.dominant_block(100, 4) == (96, 3)          # four steps need the wavefront schedule
    assert bench.dominant_block(100, 4, True) == (96, 4)
    assert bench.dominant_block(21, 3) == (15, 3)          # 19 = 5 x 3 + 2 + 2
    assert bench.dominant_block(11, 4, True) == (4, 4)      # 7 = 4 + 3, then the checked four
    assert bench.dominant_block(13, 4, True) == (4, 4)      # 9 = 4 + 3 + 2
    for ce in range(1, 40):
        for spl, wave in ((1, False), (2, False), (3, False), (4, True)):
            block, big = bench.dominant_block(ce, spl, wave)
            last = bench.check_launch_steps(ce, spl, wave)
            rest = bench.plan_plain(ce - last - block, spl, wave)
            assert bench.plan_plain(block, spl, wave) == [big] * (block // big)
            assert sorted(bench.plan_plain(block, spl, wave) + rest, reverse=True) == \
                sorted(bench.plan_plain(ce - last, spl, wave), reverse=True)


def test_kernel_hash_ignores_comments_but_not_code(bench, tmp_path):
    d = os.path.join(ROOT, "paper_2208_14870_gb300", "csrc")
    files = {n: open(os.path.join(d, n)).read()
             for n in ("lbm_core.cuh", "lbm_kernels.cuh", "lbm_ops.cuh", "lbm_step_f32.cu", "lbm_step_f16s.cu",
                       "lbm_wave_f32.cu", "lbm_wave_f16s.cu")}
    base = bench.kernel_hash(lambda n: files[n])
    assert base == bench.kernel_hash()
    commented = dict(files)
    commented["lbm_core.cuh"] = "// a new comment\n/* and a block\n comment */\n" + files["lbm_core.cuh"]
    assert bench.kernel_hash(lambda n: commented[n]) == base
    changed = dict(files)
    changed["lbm_kernels.cuh"] = files["lbm_kernels.cuh"].replace("#define LBM_BY 8", "#define LBM_BY 4")
    assert changed["lbm_kernels.cuh"] != files["lbm_kernels.cuh"]
    assert bench.kernel_hash(lambda n: changed[n]) != base
    # the field recovery is not part of the stream-collide kernels
    later = dict(files)
    later["lbm_kernels.cuh"] = files["lbm_kernels.cuh"].replace("if (out.p[4]) out.p[4][o] = -mb11 * un;",
                                                                 "if (out.p[4]) out.p[4][o] = -1.0 * mb11 * un;")
    assert later["lbm_kernels.cuh"] != files["lbm_kernels.cuh"]
    assert bench.kernel_hash(lambda n: later[n]) == base


def test_host_description(bench):
    d = bench.host_description()
    assert d["logical_cores"] >= 1 and d["machine"]
