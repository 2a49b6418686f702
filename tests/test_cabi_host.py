"""Host-side checks of the C ABI that need no GPU: the shared library loads,
exports every function include/*.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import math

import pytest

P = pytest.importorskip("paper_2208_14870_gb300")


def test_library_exports_every_declared_symbol():
    names = P.declared_functions()
    assert "lbm_create" in names and "lbm_solve" in names and "lbm_get_stress" in names
    lib = P.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_string():
    assert "sm_103a" in P.lbm_version()


@pytest.mark.parametrize("nx,ny,lam,mu,dtype", [
    (0, 4, 0.3, 0.4, P.LBM_F32),          # empty lattice
    (4, -1, 0.3, 0.4, P.LBM_F32),
    (4, 4, 0.3, 0.0, P.LBM_F64),          # mu must be > 0
    (4, 4, -0.5, 0.4, P.LBM_F64),         # lambda + mu must be > 0
    (4, 4, 0.3, 0.4, 7),                  # unknown dtype
    (4, 4, math.nan, 0.4, P.LBM_F32),
    (4, 4, 0.3, math.inf, P.LBM_F32),
    (1 << 20, 1 << 20, 0.3, 0.4, P.LBM_F32),   # more than 2^34 nodes
])
def test_create_rejects_bad_arguments(nx, ny, lam, mu, dtype):
    out = ctypes.c_void_p()
    st = P.lib().lbm_create(nx, ny, lam, mu, dtype, ctypes.byref(out))
    assert st == P.LBM_ERR_ARG
    assert out.value is None
    assert P.last_error()


def test_create_ex_rejects_bad_theta():
    out = ctypes.c_void_p()
    opt = P.lbm.lbm_options(1.5, 0.0, 0.0)
    st = P.lib().lbm_create_ex(8, 8, 0.3, 0.4, P.LBM_F32, ctypes.byref(opt), ctypes.byref(out))
    assert st == P.LBM_ERR_ARG and "theta" in P.last_error()


def test_null_context_is_rejected():
    lib = P.lib()
    assert lib.lbm_iterate(None, 1) == P.LBM_ERR_ARG
    assert lib.lbm_reset(None) == P.LBM_ERR_ARG
    assert lib.lbm_get_displacement(None, None, None) == P.LBM_ERR_ARG
    s = ctypes.c_int64()
    assert lib.lbm_get_step(None, ctypes.byref(s)) == P.LBM_ERR_ARG
    lib.lbm_destroy(None)  # ignored


def test_status_codes_match_header():
    import os
    import re
    from conftest import ROOT
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    for name, val in re.findall(r"(LBM_(?:OK|ERR_[A-Z_]+))\s*=\s*(-?\d+)", txt):
        assert getattr(P, name) == int(val)


def test_spectral_radius_matches_oracle_eigenvalues():
    """The library's Gelfand-formula spectral radius agrees with the oracle's
    numpy eigenvalues (Sec. 4 sampling)."""
    import oracle
    import oracle.fourier as F
    for E, nu, t12, t22 in ((0.082, -0.4, 0.5, 0.5), (0.11, 0.8, 0.5, 0.5), (1.0, 0.3, 0.5, 0.5),
                            (0.5, 0.2, 0.9, 0.3), (0.05, 0.999, 0.5, 0.5)):
        lam, mu = oracle.lame_2d(E, nu)
        ref = F.spectral_radius(oracle.relaxation_rates(lam, mu, tau12=t12, tau22=t22))
        got = P.lbm_spectral_radius(lam, mu, 0.0, t12, t22)
        assert abs(got - ref) < 1e-7 * ref, (E, nu, got, ref)
    with pytest.raises(P.LBMError):
        P.lbm_spectral_radius(0.3, -1.0)
