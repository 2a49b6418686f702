"""Thin ctypes binding of the C ABI in ``include/lbm.h``.

Argument marshalling only: every step of the lattice Boltzmann path runs in
the CUDA library ``_build/liblbm_gb300.so``.  There is no CPU fallback; if the
library is missing the import of this module raises.

Raw entry points keep the C names (``lbm_create``, ``lbm_iterate``, ...); they
take plain ints / floats / addresses and raise ``LBMError`` on a negative
status.  ``Lattice`` wraps one context with numpy / torch conveniences.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

LBM_F64, LBM_F32, LBM_F16S = 0, 1, 2
DTYPES = {"f64": LBM_F64, "f32": LBM_F32, "f16s": LBM_F16S}

LBM_OK = 0
LBM_ERR_ARG = -1
LBM_ERR_OOM = -2
LBM_ERR_CUDA = -3
LBM_ERR_DIVERGED = -4
LBM_ERR_NOT_CONVERGED = -5
LBM_ERR_TIMEOUT = -6
LBM_ERR_STATE = -7
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_OOM", -3: "LBM_ERR_CUDA",
                -4: "LBM_ERR_DIVERGED", -5: "LBM_ERR_NOT_CONVERGED", -6: "LBM_ERR_TIMEOUT",
                -7: "LBM_ERR_STATE"}


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(status, "?"), status, message))
        self.status = status


class lbm_options(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("tau12", ctypes.c_double), ("tau22", ctypes.c_double)]


class lbm_rates(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("w11", "ws", "wd", "w12", "w21", "w22", "theta")]


_c = ctypes
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_SIGS = {
    "lbm_create": (_c.c_int, [_c.c_int, _c.c_int, _c.c_double, _c.c_double, _c.c_int, _c.POINTER(_vp)]),
    "lbm_create_ex": (_c.c_int, [_c.c_int, _c.c_int, _c.c_double, _c.c_double, _c.c_int,
                                 _c.POINTER(lbm_options), _c.POINTER(_vp)]),
    "lbm_destroy": (None, [_vp]),
    "lbm_set_stream": (_c.c_int, [_vp, _vp]),
    "lbm_set_host_transfer": (_c.c_int, [_vp, _c.c_int]),
    "lbm_get_host_transfer": (_c.c_int, [_vp, _c.POINTER(_c.c_int)]),
    "lbm_set_steps_per_launch": (_c.c_int, [_vp, _c.c_int]),
    "lbm_get_steps_per_launch": (_c.c_int, [_vp, _c.POINTER(_c.c_int)]),
    "lbm_set_wavefront": (_c.c_int, [_vp, _c.c_int]),
    "lbm_get_wavefront": (_c.c_int, [_vp, _c.POINTER(_c.c_int)]),
    "lbm_set_force": (_c.c_int, [_vp, _vp, _vp]),
    "lbm_set_force_device": (_c.c_int, [_vp, _vp, _vp]),
    "lbm_set_force_corrected": (_c.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_spectral_radius": (_c.c_int, [_c.c_double, _c.c_double, _c.c_double, _c.c_double,
                                       _c.c_double, _c.c_int, _c.c_int, _c.POINTER(_c.c_double)]),
    "lbm_error_constants": (_c.c_int, [_c.c_double, _c.c_double, _c.c_double, _c.c_double,
                                       _c.c_double, _vp]),
    "lbm_error_constants_scheme": (_c.c_int, [_c.c_double, _c.c_double, _c.c_double, _c.c_double,
                                              _c.c_double, _vp]),
    "lbm_fourth_order_taus": (_c.c_int, [_c.c_double, _c.c_double, _c.c_double,
                                         _c.POINTER(_c.c_double), _c.POINTER(_c.c_double)]),
    "lbm_reset": (_c.c_int, [_vp]),
    "lbm_iterate": (_c.c_int, [_vp, _i64]),
    "lbm_iterate_checked": (_c.c_int, [_vp, _i64, _c.c_int, _vp]),
    "lbm_solve": (_c.c_int, [_vp, _c.c_double, _i64, _c.c_int, _c.POINTER(_i64),
                             _c.POINTER(_c.c_double)]),
    "lbm_get_displacement": (_c.c_int, [_vp, _vp, _vp]),
    "lbm_get_stress": (_c.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_get_fields_device": (_c.c_int, [_vp, _vp]),
    "lbm_get_populations": (_c.c_int, [_vp, _vp]),
    "lbm_set_populations": (_c.c_int, [_vp, _vp]),
    "lbm_get_step": (_c.c_int, [_vp, _c.POINTER(_i64)]),
    "lbm_get_rates": (_c.c_int, [_vp, _c.POINTER(lbm_rates)]),
    "lbm_get_device_bytes": (_c.c_int, [_vp, _c.POINTER(_c.c_size_t)]),
    "lbm_last_error": (_c.c_char_p, []),
    "lbm_fp64_fma_rate": (_c.c_int, [_c.POINTER(_c.c_double)]),
    "lbm_step_checked_noalloc": (_c.c_int, [_c.c_int, _c.c_int, _c.c_double, _c.c_double, _c.c_int,
                                            _vp, _vp, _vp, _vp, _vp, _vp, _c.c_int, _vp]),
    "lbm_version": (_c.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def _load() -> ctypes.CDLL:
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("CUDA library %s is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def last_error() -> str:
    return _lib.lbm_last_error().decode()


def _check(status: int, what: str) -> int:
    if status != LBM_OK:
        raise LBMError(status, "%s: %s" % (what, last_error()))
    return status


# ---------------------------------------------------------------------------
# Raw entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def lbm_create(nx: int, ny: int, lam: float, mu: float, dtype: int) -> int:
    out = _vp()
    _check(_lib.lbm_create(nx, ny, lam, mu, dtype, ctypes.byref(out)), "lbm_create")
    return out.value


def lbm_create_ex(nx, ny, lam, mu, dtype, theta=0.0, tau12=0.0, tau22=0.0) -> int:
    out = _vp()
    opt = lbm_options(theta, tau12, tau22)
    _check(_lib.lbm_create_ex(nx, ny, lam, mu, dtype, ctypes.byref(opt), ctypes.byref(out)),
           "lbm_create_ex")
    return out.value


def lbm_destroy(ctx: int) -> None:
    _lib.lbm_destroy(ctx)


def lbm_set_stream(ctx: int, stream: int) -> None:
    _check(_lib.lbm_set_stream(ctx, stream), "lbm_set_stream")


def lbm_set_host_transfer(ctx: int, mode: int) -> None:
    _check(_lib.lbm_set_host_transfer(ctx, mode), "lbm_set_host_transfer")


def lbm_get_host_transfer(ctx: int) -> int:
    m = _c.c_int()
    _check(_lib.lbm_get_host_transfer(ctx, _c.byref(m)), "lbm_get_host_transfer")
    return m.value


def lbm_set_steps_per_launch(ctx: int, k: int) -> None:
    _check(_lib.lbm_set_steps_per_launch(ctx, k), "lbm_set_steps_per_launch")


def lbm_get_steps_per_launch(ctx: int) -> int:
    k = _c.c_int()
    _check(_lib.lbm_get_steps_per_launch(ctx, _c.byref(k)), "lbm_get_steps_per_launch")
    return k.value


def lbm_set_wavefront(ctx: int, rows: int) -> None:
    _check(_lib.lbm_set_wavefront(ctx, rows), "lbm_set_wavefront")


def lbm_get_wavefront(ctx: int) -> int:
    r = _c.c_int()
    _check(_lib.lbm_get_wavefront(ctx, _c.byref(r)), "lbm_get_wavefront")
    return r.value


def lbm_set_force(ctx: int, gx_ptr: int, gy_ptr: int) -> None:
    _check(_lib.lbm_set_force(ctx, gx_ptr, gy_ptr), "lbm_set_force")


def lbm_set_force_device(ctx: int, gx_ptr: int, gy_ptr: int) -> None:
    _check(_lib.lbm_set_force_device(ctx, gx_ptr, gy_ptr), "lbm_set_force_device")


def lbm_set_force_corrected(ctx: int, gx_ptr: int, gy_ptr: int, d_ptr: int) -> None:
    _check(_lib.lbm_set_force_corrected(ctx, gx_ptr, gy_ptr, d_ptr), "lbm_set_force_corrected")


def lbm_error_constants(E: float, nu: float, theta: float = 0.0, tau12: float = 0.0,
                        tau22: float = 0.0) -> np.ndarray:
    """[C1..C5, D1..D3] as printed in Appendix B."""
    out = np.zeros(8)
    _check(_lib.lbm_error_constants(E, nu, theta, tau12, tau22, out.ctypes.data),
           "lbm_error_constants")
    return out


def lbm_error_constants_scheme(E: float, nu: float, theta: float = 0.0, tau12: float = 0.0,
                               tau22: float = 0.0) -> np.ndarray:
    """[C1..C5, D1..D3] of the scheme (Appendix B with three misprints read)."""
    out = np.zeros(8)
    _check(_lib.lbm_error_constants_scheme(E, nu, theta, tau12, tau22, out.ctypes.data),
           "lbm_error_constants_scheme")
    return out


def lbm_fourth_order_taus(E: float, nu: float, theta: float = 0.0) -> tuple[float, float]:
    """(tau12, tau22) zeroing C5 and C1 (fourth-order special case)."""
    t12, t22 = _c.c_double(), _c.c_double()
    _check(_lib.lbm_fourth_order_taus(E, nu, theta, _c.byref(t12), _c.byref(t22)), "lbm_fourth_order_taus")
    return t12.value, t22.value


def lbm_spectral_radius(lam: float, mu: float, theta: float = 0.0, tau12: float = 0.0,
                        tau22: float = 0.0, nk: int = 50, nphi: int = 5) -> float:
    """Sampled sup of the von Neumann spectral radius (<= 1: stable)."""
    rho = ctypes.c_double()
    st = _lib.lbm_spectral_radius(lam, mu, theta, tau12, tau22, nk, nphi, ctypes.byref(rho))
    if st != LBM_OK:
        raise LBMError(st, "lbm_spectral_radius: invalid parameters")
    return rho.value


def lbm_reset(ctx: int) -> None:
    _check(_lib.lbm_reset(ctx), "lbm_reset")


def lbm_iterate(ctx: int, n: int) -> None:
    _check(_lib.lbm_iterate(ctx, n), "lbm_iterate")


def lbm_iterate_checked(ctx: int, n: int, check_every: int, out_ptr: Optional[int] = None) -> None:
    _check(_lib.lbm_iterate_checked(ctx, n, check_every, out_ptr), "lbm_iterate_checked")


def lbm_solve(ctx: int, tol: float, max_iters: int, check_every: int):
    """Returns (status, iters, residual); LBM_ERR_NOT_CONVERGED and
    LBM_ERR_DIVERGED are returned, other errors raise."""
    it = _i64()
    r = ctypes.c_double()
    st = _lib.lbm_solve(ctx, tol, max_iters, check_every, ctypes.byref(it), ctypes.byref(r))
    if st not in (LBM_OK, LBM_ERR_NOT_CONVERGED, LBM_ERR_DIVERGED):
        _check(st, "lbm_solve")
    return st, it.value, r.value


def lbm_get_displacement(ctx: int, ux_ptr: int, uy_ptr: int) -> None:
    _check(_lib.lbm_get_displacement(ctx, ux_ptr, uy_ptr), "lbm_get_displacement")


def lbm_get_stress(ctx: int, sxx_ptr: int, syy_ptr: int, sxy_ptr: int) -> None:
    _check(_lib.lbm_get_stress(ctx, sxx_ptr, syy_ptr, sxy_ptr), "lbm_get_stress")


def lbm_get_fields_device(ctx: int, out_ptr: int) -> None:
    _check(_lib.lbm_get_fields_device(ctx, out_ptr), "lbm_get_fields_device")


def lbm_get_populations(ctx: int, f_ptr: int) -> None:
    _check(_lib.lbm_get_populations(ctx, f_ptr), "lbm_get_populations")


def lbm_set_populations(ctx: int, f_ptr: int) -> None:
    _check(_lib.lbm_set_populations(ctx, f_ptr), "lbm_set_populations")


def lbm_get_step(ctx: int) -> int:
    s = _i64()
    _check(_lib.lbm_get_step(ctx, ctypes.byref(s)), "lbm_get_step")
    return s.value


def lbm_get_rates(ctx: int) -> dict:
    r = lbm_rates()
    _check(_lib.lbm_get_rates(ctx, ctypes.byref(r)), "lbm_get_rates")
    return {k: getattr(r, k) for k, _ in lbm_rates._fields_}


def lbm_get_device_bytes(ctx: int) -> int:
    b = ctypes.c_size_t()
    _check(_lib.lbm_get_device_bytes(ctx, ctypes.byref(b)), "lbm_get_device_bytes")
    return b.value


LBM_NOALLOC_MAX_BLOCKS = 1024
LBM_TILE_TWO_STEP = 3
LBM_TILE_WAVE = 5
LBM_HOST_DIRECT = 0
LBM_HOST_COPY = 1


def lbm_step_checked_noalloc(nx: int, ny: int, lam: float, mu: float, dtype: int, f_src: int,
                             f_dst: int, gx: int, gy: int, snapshot: int, result: int,
                             grid_blocks: int = 0, stream: int = 0) -> None:
    """One residual-checked step on caller-owned device buffers; allocates
    nothing (see include/lbm.h).  Raises LBMError on a rejected call."""
    st = _lib.lbm_step_checked_noalloc(nx, ny, lam, mu, dtype, f_src, f_dst, gx, gy, snapshot,
                                       result, grid_blocks, stream)
    if st != LBM_OK:
        raise LBMError(st, "lbm_step_checked_noalloc rejected the call (needs LBM_F64 or "
                           "LBM_F32, 1 <= nx, ny, nx*ny <= 2^31, mu > 0, lambda + mu > 0, "
                           "non-null distinct buffers, 0 <= grid_blocks <= %d)"
                       % LBM_NOALLOC_MAX_BLOCKS)


def lbm_fp64_fma_rate() -> float:
    """Measured FP64 FMA throughput of the current device (G thread-level
    FP64 instructions per second)."""
    r = ctypes.c_double()
    _check(_lib.lbm_fp64_fma_rate(ctypes.byref(r)), "lbm_fp64_fma_rate")
    return r.value


def lbm_version() -> str:
    return _lib.lbm_version().decode()


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

def _host_f64(a: np.ndarray, n: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


class Lattice:
    """One periodic lattice (context) on the current CUDA device."""

    def __init__(self, nx: int, ny: int, lam: float, mu: float, dtype: str = "f32",
                 theta: float = 0.0, tau12: float = 0.0, tau22: float = 0.0,
                 check_stability: bool = False):
        self.nx, self.ny, self.dtype = int(nx), int(ny), dtype
        if check_stability:
            rho = lbm_spectral_radius(lam, mu, theta, tau12, tau22)
            if rho > 1.0 + 1e-9:
                import warnings
                warnings.warn("lattice Boltzmann parameters are von Neumann unstable "
                              "(spectral radius %.6f > 1)" % rho, RuntimeWarning)
        self.ctx = lbm_create_ex(self.nx, self.ny, float(lam), float(mu), DTYPES[dtype],
                                 theta, tau12, tau22)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n(self) -> int:
        return self.nx * self.ny

    def set_stream(self, stream_handle: int):
        lbm_set_stream(self.ctx, stream_handle)

    @property
    def host_transfer(self) -> int:
        return lbm_get_host_transfer(self.ctx)

    @host_transfer.setter
    def host_transfer(self, mode: int):
        lbm_set_host_transfer(self.ctx, mode)

    def set_force(self, gx, gy):
        """Host numpy arrays (copied) or device torch tensors (float64)."""
        if hasattr(gx, "is_cuda") and gx.is_cuda:
            assert gx.dtype == gy.dtype and str(gx.dtype) == "torch.float64"
            assert gx.is_contiguous() and gy.is_contiguous() and gx.numel() == self.n
            lbm_set_force_device(self.ctx, gx.data_ptr(), gy.data_ptr())
            return
        gxh, gyh = _host_f64(gx, self.n), _host_f64(gy, self.n)
        lbm_set_force(self.ctx, gxh.ctypes.data, gyh.ctypes.data)

    def set_force_corrected(self, gx, gy, d):
        """Host force with the higher-order correction (D1, D2, D3) applied on the device."""
        gxh, gyh = _host_f64(gx, self.n), _host_f64(gy, self.n)
        dd = np.ascontiguousarray(d, dtype=np.float64)
        assert dd.shape == (3,)
        lbm_set_force_corrected(self.ctx, gxh.ctypes.data, gyh.ctypes.data, dd.ctypes.data)

    def reset(self):
        lbm_reset(self.ctx)

    def iterate(self, n: int):
        lbm_iterate(self.ctx, int(n))

    def iterate_checked(self, n: int, check_every: int) -> np.ndarray:
        out = np.zeros(5, dtype=np.float64)
        lbm_iterate_checked(self.ctx, int(n), int(check_every), out.ctypes.data)
        return out

    def solve(self, tol: float, max_iters: int = 10_000_000, check_every: int = 100):
        return lbm_solve(self.ctx, float(tol), int(max_iters), int(check_every))

    def displacement(self) -> np.ndarray:
        out = np.empty((2, self.ny, self.nx), dtype=np.float64)
        lbm_get_displacement(self.ctx, out[0].ctypes.data, out[1].ctypes.data)
        return out

    def stress(self) -> np.ndarray:
        out = np.empty((3, self.ny, self.nx), dtype=np.float64)
        lbm_get_stress(self.ctx, out[0].ctypes.data, out[1].ctypes.data, out[2].ctypes.data)
        return out

    def fields(self) -> np.ndarray:
        """[u_x, u_y, sigma_xx, sigma_yy, sigma_xy] (lattice units), host FP64."""
        return np.concatenate([self.displacement(), self.stress()])

    def fields_device(self, out):
        """Write the five fields into a contiguous CUDA float64 tensor of 5*n."""
        assert out.is_cuda and out.is_contiguous() and out.numel() == 5 * self.n
        lbm_get_fields_device(self.ctx, out.data_ptr())
        return out

    def populations(self) -> np.ndarray:
        out = np.empty((8, self.ny, self.nx), dtype=np.float64)
        lbm_get_populations(self.ctx, out.ctypes.data)
        return out

    def set_populations(self, f: np.ndarray):
        f = _host_f64(f, 8 * self.n)
        lbm_set_populations(self.ctx, f.ctypes.data)

    @property
    def step(self) -> int:
        return lbm_get_step(self.ctx)

    @property
    def steps_per_launch(self) -> int:
        return lbm_get_steps_per_launch(self.ctx)

    @steps_per_launch.setter
    def steps_per_launch(self, k: int):
        lbm_set_steps_per_launch(self.ctx, k)

    @property
    def wavefront(self) -> int:
        """Rows per block segment of the wavefront schedule (-1: chosen per
        launch, 0: tile schedule)."""
        return lbm_get_wavefront(self.ctx)

    @wavefront.setter
    def wavefront(self, rows: int):
        lbm_set_wavefront(self.ctx, rows)

    @property
    def rates(self) -> dict:
        return lbm_get_rates(self.ctx)

    @property
    def device_bytes(self) -> int:
        return lbm_get_device_bytes(self.ctx)


def declared_functions(header: Optional[str] = None) -> list[str]:
    """Names of the functions declared in include/*.h."""
    import glob
    import re
    inc = os.path.dirname(header) if header else _build.INCLUDE
    names = []
    for h in sorted(glob.glob(os.path.join(inc, "*.h"))):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


# ---------------------------------------------------------------------------
# Batched solves (lbm_batch_solve)
# ---------------------------------------------------------------------------

class lbm_problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("lam", ctypes.c_double),
                ("mu", ctypes.c_double), ("gx", _vp), ("gy", _vp)]


class lbm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int64), ("residual", ctypes.c_double),
                ("ux", _vp), ("uy", _vp), ("sxx", _vp), ("syy", _vp), ("sxy", _vp),
                ("transposed", ctypes.c_int)]


class lbm_batch_report(ctypes.Structure):
    _fields_ = [("tile_v", ctypes.c_int), ("blocks", ctypes.c_int), ("chunks", ctypes.c_int64),
                ("lattice_updates", ctypes.c_int64), ("device_ms", ctypes.c_double),
                ("wall_ms", ctypes.c_double)]


_lib.lbm_batch_solve.restype = ctypes.c_int
_lib.lbm_batch_solve.argtypes = [ctypes.c_int, ctypes.POINTER(lbm_problem), ctypes.c_int,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_int64,
                                 ctypes.POINTER(lbm_result), ctypes.POINTER(lbm_batch_report)]


def batch_solve(problems, dtype: str = "f32", tol: float = 1e-8, check_every: int = 100,
                max_iters: int = 10_000_000, fields: bool = True):
    """Solve many problems in one arena.  ``problems``: iterable of
    (nx, ny, lam, mu, gx, gy) with host FP64 arrays.  Returns (results, report):
    results is a list of dicts (status, iters, residual, transposed[, fields
    (5, ny, nx)])."""
    problems = list(problems)
    cnt = len(problems)
    arr = (lbm_problem * cnt)()
    res = (lbm_result * cnt)()
    keep = []
    outs = []
    for i, (nx, ny, lam, mu, gx, gy) in enumerate(problems):
        gxh = _host_f64(gx, nx * ny)
        gyh = _host_f64(gy, nx * ny)
        keep += [gxh, gyh]
        arr[i] = lbm_problem(nx, ny, lam, mu, gxh.ctypes.data, gyh.ctypes.data)
        if fields:
            o = np.empty((5, ny, nx), dtype=np.float64)
            outs.append(o)
            res[i].ux, res[i].uy, res[i].sxx, res[i].syy, res[i].sxy = [o[c].ctypes.data for c in range(5)]
        else:
            outs.append(None)
    rep = lbm_batch_report()
    _check(_lib.lbm_batch_solve(cnt, arr, DTYPES[dtype], tol, check_every, max_iters, res,
                                ctypes.byref(rep)), "lbm_batch_solve")
    results = []
    for i in range(cnt):
        d = {"status": res[i].status, "iters": res[i].iters, "residual": res[i].residual,
             "transposed": bool(res[i].transposed)}
        if fields:
            d["fields"] = outs[i]
        results.append(d)
    report = {k: getattr(rep, k) for k, _ in lbm_batch_report._fields_}
    return results, report


# ---------------------------------------------------------------------------
# Continuous-batching server (lbm_server_*)
# ---------------------------------------------------------------------------

LBM_PENDING = 1


class lbm_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p95_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("lattice_updates", ctypes.c_int64),
                ("device_ms", ctypes.c_double), ("chunks", ctypes.c_int64),
                ("hbm_bytes", ctypes.c_size_t), ("peak_running", ctypes.c_int),
                ("tile_v", ctypes.c_int), ("failed", ctypes.c_int),
                ("memory_waits", ctypes.c_int64), ("peak_resident_bytes", ctypes.c_size_t)]


for _name, _res, _args in (
        ("lbm_server_create", ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_vp)]),
        ("lbm_server_destroy", None, [_vp]),
        ("lbm_server_submit", ctypes.c_int, [_vp, ctypes.POINTER(lbm_problem), ctypes.c_int,
                                             ctypes.c_double, ctypes.c_int64,
                                             ctypes.POINTER(ctypes.c_uint64)]),
        ("lbm_server_poll", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(lbm_result)]),
        ("lbm_server_wait", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double,
                                           ctypes.POINTER(lbm_result)]),
        ("lbm_server_cancel", ctypes.c_int, [_vp, ctypes.c_uint64]),
        ("lbm_server_stats", ctypes.c_int, [_vp, ctypes.POINTER(lbm_stats)])):
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class Server:
    """Continuous-batching solve server on the current CUDA device."""

    def __init__(self, hbm_budget_bytes: int, check_every: int = 100):
        out = _vp()
        _check(_lib.lbm_server_create(int(hbm_budget_bytes), int(check_every), ctypes.byref(out)),
               "lbm_server_create")
        self.srv = out.value
        self._shapes = {}

    def close(self):
        if getattr(self, "srv", None):
            _lib.lbm_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, nx, ny, lam, mu, gx, gy, dtype="f32", tol=1e-8, max_iters=10_000_000) -> int:
        gxh = _host_f64(gx, nx * ny)
        gyh = _host_f64(gy, nx * ny)
        prob = lbm_problem(nx, ny, lam, mu, gxh.ctypes.data, gyh.ctypes.data)
        t = ctypes.c_uint64()
        _check(_lib.lbm_server_submit(self.srv, ctypes.byref(prob), DTYPES[dtype], tol, max_iters,
                                      ctypes.byref(t)), "lbm_server_submit")
        self._shapes[t.value] = (nx, ny)
        return t.value

    def _result(self, fn, ticket, *extra, fields=True):
        if ticket not in self._shapes:  # let the library reject it
            _check(fn(self.srv, ticket, *extra, None), fn.__name__)
        nx, ny = self._shapes[ticket]
        res = lbm_result()
        out = None
        if fields:
            out = np.empty((5, ny, nx), dtype=np.float64)
            res.ux, res.uy, res.sxx, res.syy, res.sxy = [out[c].ctypes.data for c in range(5)]
        st = fn(self.srv, ticket, *extra, ctypes.byref(res))
        if st == LBM_PENDING:
            return None
        _check(st, fn.__name__)
        del self._shapes[ticket]
        d = {"status": res.status, "iters": res.iters, "residual": res.residual,
             "transposed": bool(res.transposed)}
        if fields:
            d["fields"] = out
        return d

    def poll(self, ticket: int, fields: bool = True):
        return self._result(_lib.lbm_server_poll, ticket, fields=fields)

    def wait(self, ticket: int, timeout_s: float = 600.0, fields: bool = True):
        return self._result(_lib.lbm_server_wait, ticket, ctypes.c_double(timeout_s), fields=fields)

    def cancel(self, ticket: int):
        _check(_lib.lbm_server_cancel(self.srv, ticket), "lbm_server_cancel")
        self._shapes.pop(ticket, None)

    def stats(self) -> dict:
        s = lbm_stats()
        _check(_lib.lbm_server_stats(self.srv, ctypes.byref(s)), "lbm_server_stats")
        return {k: getattr(s, k) for k, _ in lbm_stats._fields_}
