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


def simulate_launches(iters, check_every, spl):
    """Launch sequence of lbm_iterate_checked from step 0, written out launch
    by launch as the library plans it: plain steps grouped into launches of spl
    steps, leftovers in launches of 2 or 1, and a check step (index + 1 a
    multiple of check_every) as the last step of a launch of at most two
    steps."""
    def plain(m):
        count = 0
        while m > 0:
            k = min(spl, m)
            if spl == 3 and m == 4:
                k = 2          # 4 = 2 + 2 instead of 3 + 1
            m -= k
            count += 1
        return count
    launches, step, left = 0, 0, iters
    while left > 0:
        to_check = check_every - step % check_every
        if to_check > left:
            launches += plain(left)
            break
        last = min(spl, 2, to_check)      # the check rides on a launch of at most two steps
        launches += plain(to_check - last) + 1
        step += to_check
        left -= to_check
    return launches


@pytest.mark.parametrize("spl", [1, 2, 3])
def test_launch_count_matches_the_schedule(bench, spl):
    for iters in (0, 1, 2, 7, 99, 100, 101, 1000, 1234):
        for ce in (1, 2, 3, 7, 10, 100):
            assert bench.launches_per_iterate(iters, ce, spl) == simulate_launches(iters, ce, spl), (iters, ce)
    assert bench.launches_per_iterate(1000, 100, 2) == 500
    assert bench.launches_per_iterate(1000, 100, 1) == 1000
    assert bench.launches_per_iterate(1000, 100, 3) == 10 * (33 + 1)   # 98 = 32 x 3 + 2, then the check pair


def test_kernel_hash_ignores_comments_but_not_code(bench, tmp_path):
    d = os.path.join(ROOT, "paper_2208_14870_gb300", "csrc")
    files = {n: open(os.path.join(d, n)).read()
             for n in ("lbm_core.cuh", "lbm_kernels.cuh", "lbm_ops.cuh", "lbm_step_f32.cu", "lbm_step_f16s.cu")}
    base = bench.kernel_hash(lambda n: files[n])
    assert base == bench.kernel_hash()
    commented = dict(files)
    commented["lbm_core.cuh"] = "// a new comment\n/* and a block\n comment */\n" + files["lbm_core.cuh"]
    assert bench.kernel_hash(lambda n: commented[n]) == base
    changed = dict(files)
    changed["lbm_kernels.cuh"] = files["lbm_kernels.cuh"].replace("#define LBM_BY 8", "#define LBM_BY 4")
    assert changed["lbm_kernels.cuh"] != files["lbm_kernels.cuh"]
    assert bench.kernel_hash(lambda n: changed[n]) != base


def test_host_description(bench):
    d = bench.host_description()
    assert d["logical_cores"] >= 1 and d["machine"]
