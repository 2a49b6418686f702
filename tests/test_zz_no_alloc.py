"""The allocation-free residual-checked step, lbm_step_checked_noalloc.

It is for callers that may not allocate device memory (plug-ins whose host
application owns all device memory, latency-critical loops that cannot pay
for cudaMalloc / cudaFree).  It runs the same kernel as the context API's
lbm_iterate_checked with its reduction scratch in a static device array, so
two calls in a row must reproduce, through the C ABI, what two residual-checked
steps of a context give: the same populations and the same residual numbers
within the FP64 tolerance of the parity tests (1e-12 relative) -- with the
default grid, with 3 blocks (many tiles per block, a three-slot last-block
reduction) and with the largest grid the static scratch allows.

The snapshot is 16 bytes per node for both storage types (two planes of
doubles, or of (hi, lo) float pairs).

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2208_14870_gb300 as P  # noqa: E402

CX = [1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 1, 0, -1, 1, 1, -1, -1]
TOL = 1e-12


def stored_to_pre_collision(fstar):
    """The stored state holds f*_i(x); the pre-collision populations are
    f_i(x) = f*_i(x - c_i)."""
    return np.stack([np.roll(fstar[i], shift=(CY[i], CX[i]), axis=(0, 1)) for i in range(8)])


def rel(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


@pytest.mark.parametrize("grid", [0, 3, P.LBM_NOALLOC_MAX_BLOCKS])
# (1024 x 1040 FP32 has 1040 tiles of 128 x 8 nodes: the largest grid is
# 1024 blocks, some of which take two tiles)
@pytest.mark.parametrize("dtype,nx,ny", [("f32", 300, 200), ("f64", 97, 61), ("f32", 1024, 1040)])
def test_noalloc_step_matches_context_api_twice(dtype, nx, ny, grid):
    lam, mu = W.lame_2d(1.0, 0.3)
    pw = W.random_force(nx, ny, 6, 4, seed=77)
    gx, gy = W.random_force_grid(pw)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    code = P.DTYPES[dtype]

    # Context API: two residual-checked steps (check every step).
    ref_state, ref_res = [], []
    with P.Lattice(nx, ny, lam, mu, dtype) as lat:
        lat.set_force(gx, gy)
        for _ in range(2):
            ref_res.append(lat.iterate_checked(1, 1))
            ref_state.append(lat.populations())

    # Caller-owned buffers, no allocation inside the library.
    n = nx * ny
    f_a = torch.zeros(8 * n, dtype=tdt, device="cuda")
    f_b = torch.zeros(8 * n, dtype=tdt, device="cuda")
    gxd = torch.from_numpy(gx).to(device="cuda", dtype=tdt).contiguous()
    gyd = torch.from_numpy(gy).to(device="cuda", dtype=tdt).contiguous()
    snap = torch.zeros(2 * n, dtype=torch.float64, device="cuda")   # 16 bytes per node
    result = torch.zeros(5, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    bufs = [(f_a, f_b), (f_b, f_a)]
    for k in range(2):
        src, dst = bufs[k]
        P.lbm_step_checked_noalloc(nx, ny, lam, mu, code, src.data_ptr(), dst.data_ptr(),
                                   gxd.data_ptr(), gyd.data_ptr(), snap.data_ptr(),
                                   result.data_ptr(), grid, stream)
        torch.cuda.synchronize()
        raw = result.cpu().numpy()
        fstar = dst.double().cpu().numpy().reshape(8, ny, nx)
        assert rel(stored_to_pre_collision(fstar), ref_state[k]) < TOL
        # max|u| and ||u||_2 of this step's input state
        assert abs(raw[1] - ref_res[k][2]) <= TOL * ref_res[k][2]
        assert abs(np.sqrt(raw[3]) - ref_res[k][3]) <= TOL * ref_res[k][3]
        assert raw[4] == 0.0
        if k == 1:
            # second call: window of one step, r_inf and r_2 as the context reports them
            r_inf = raw[0] / raw[1]
            r_2 = np.sqrt(raw[2]) / np.sqrt(raw[3])
            assert abs(r_inf - ref_res[k][0]) <= TOL * ref_res[k][0]
            assert abs(r_2 - ref_res[k][1]) <= TOL * ref_res[k][1]


def test_noalloc_rejects_more_blocks_than_its_scratch_holds():
    lam, mu = W.lame_2d(1.0, 0.3)
    nx = ny = 64
    f_a = torch.zeros(8 * nx * ny, device="cuda")
    f_b = torch.zeros(8 * nx * ny, device="cuda")
    g = torch.zeros(nx * ny, device="cuda")
    snap = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")   # 16 bytes per node
    result = torch.zeros(5, dtype=torch.float64, device="cuda")
    args = [nx, ny, lam, mu, P.LBM_F32, f_a.data_ptr(), f_b.data_ptr(), g.data_ptr(),
            g.data_ptr(), snap.data_ptr(), result.data_ptr()]
    lib = P.lib()
    assert lib.lbm_step_checked_noalloc(*args, P.LBM_NOALLOC_MAX_BLOCKS + 1, None) == P.LBM_ERR_ARG
    with pytest.raises(P.LBMError, match="grid_blocks"):
        P.lbm_step_checked_noalloc(*args, P.LBM_NOALLOC_MAX_BLOCKS + 1)
    bad = list(args)
    bad[4] = P.LBM_F16S
    assert lib.lbm_step_checked_noalloc(*bad, 0, None) == P.LBM_ERR_ARG
    # an explicit grid within the limit is accepted
    assert lib.lbm_step_checked_noalloc(*args, 3, None) == P.LBM_OK
    torch.cuda.synchronize()
