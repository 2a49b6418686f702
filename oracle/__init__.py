"""FP64 CPU oracle for the periodic lattice Boltzmann scheme for linear elasticity
(Boolakee, Geier, De Lorenzis, arXiv 2208.14870).

TEST INFRASTRUCTURE ONLY.  The oracle exists to check the CUDA library; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path and never
imports the library package.

Parts:
  * ``lbm_oracle.c`` (loaded here through ctypes): one pseudo-time step as
    the composition of the defining equations, node by node in plain C, FP64
    -- the raw-moment map (Eq. moments, Eq. replace_raw), the collision of
    Eq. collision on the moments with the Table 1 equilibria and the force
    split around it (Eqs. coll10/coll01 and coll10post/coll01post), the
    populations from Eq. moments_post, streaming (Eq. streaming) with the
    periodic wrap of Sec. 5.1 -- and the solution fields of Table 2.
  * this module: the relaxation rates tied to the Lame parameters (Table 1,
    Eqs. match11/matchd/matchs, Eq. relaxation_rate), the 2D material
    relations (Eq. material_relations), the pseudo-time loop to steady state
    (Sec. 2.1: iterate until the change of u is below a tolerance) and the
    grid norms of Sec. 6.1.
  * ``fourier.py``: the one-step operator of Eq. lbmvector, its von Neumann
    spectral radius (Sec. 4), and the exact discrete steady state mode by
    mode.

  * Sec. 4 / Appendices B and C helpers: the printed error constants and
    their read form, the finite-difference force correction, the exact
    discrete leading error (axis-aligned modes, and every constant of
    Appendix B from the one-step operator), and the relaxation times of the
    fourth-order case.

Every function here is pinned by ``tests/test_oracle_*.py`` against the
paper's printed values, closed forms, brute force on small lattices and exact
invariants.  The constants of Appendix B are pinned one by one against the
scheme's exact discrete leading error (``leading_error_exact``, extracted
from the one-step operator), which shows three misprints (C2, D1, D2, applied
in ``error_constants_read``) and a fourth one in Appendix C's tau_22
(``fourth_order_taus_scheme``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "liblbm_oracle.so")
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_lock = threading.Lock()
_lib = None

THETA_STANDARD = 1.0 / 3.0  # Sec. 3.3.2 (isotropy argument), Table 1


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` into ``oracle/_build/liblbm_oracle.so`` (gcc, -O2,
    no FMA contraction).  Returns the path of the shared object."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call([
            "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
            "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                       dp, ctypes.c_long, dp, dp]
            lib.oracle_collide.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                           dp, dp, dp]
            lib.oracle_moments.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
            lib.oracle_fields.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                          dp, dp]
            lib.oracle_raw_moment_inverse.argtypes = [ctypes.c_int, dp]
            for fn in (lib.oracle_run, lib.oracle_collide, lib.oracle_moments,
                       lib.oracle_fields, lib.oracle_raw_moment_inverse):
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ----------------------------------------------------------------------------
# Material parameters and relaxation rates
# ----------------------------------------------------------------------------

def lame_2d(E: float, nu: float) -> tuple[float, float]:
    """Lame parameters of the 2D (not plane-strain) medium, Eq. material_relations:
    lambda = E nu / (1 - nu^2), mu = E / (2 (1 + nu))."""
    return E * nu / (1.0 - nu * nu), E / (2.0 * (1.0 + nu))


def relaxation_rates(lam: float, mu: float, theta: float = THETA_STANDARD,
                     tau12: float = 0.5, tau22: float = 0.5) -> np.ndarray:
    """Rates [w_11, w_s, w_d, w_12, w_21, w_22, theta] in lattice units.

    Table 1 / Eqs. match11, matchd, matchs: theta*tau_11 = mu,
    (1 - theta)/2 * tau_d = mu, (1 + theta)/2 * tau_s = K with K = lambda + mu
    (Eq. material_relations); tau_12 = tau_21 and tau_22 default to 1/2
    (Sec. 3.3.2, last remarks).  Eq. relaxation_rate: w = 1 / (tau + 1/2).
    """
    K = lam + mu
    tau11 = mu / theta
    tau_d = 2.0 * mu / (1.0 - theta)
    tau_s = 2.0 * K / (1.0 + theta)
    w = [1.0 / (t + 0.5) for t in (tau11, tau_s, tau_d, tau12, tau12, tau22)]
    return np.array(w + [theta], dtype=np.float64)


def fourth_order_taus(lam: float, mu: float, theta: float = THETA_STANDARD) -> tuple[float, float]:
    """tau_12 = tau_21 and tau_22 of the fourth-order special case (Appendix C)."""
    K = lam + mu
    t11 = mu / theta
    td = 2.0 * mu / (1.0 - theta)
    ts = 2.0 * K / (1.0 + theta)
    tau12 = (2.0 - 3.0 * theta + 12.0 * theta * t11 ** 2) / (12.0 * (1.0 - theta) * t11)
    num = ((1.0 - theta) * td + (1.0 + theta) * ts) * (
        theta * (2.0 - 3.0 * theta) * (ts - td) - 12.0 * theta ** 2 * t11 ** 2 * (ts - td)
        + 2.0 * t11 * (1.0 - theta - 6.0 * (1.0 - theta) ** 2 * td ** 2
                       - 6.0 * (1.0 - theta ** 2) * ts ** 2))
    den = 2.0 * theta * (2.0 - 3.0 * theta + 12.0 * theta * t11 ** 2) * (ts - td)
    return tau12, num / den


def fourth_order_taus_scheme(lam: float, mu: float, theta: float = THETA_STANDARD) -> tuple[float, float]:
    """tau_12 = tau_21 and tau_22 that zero both C5 and C1 of this scheme
    (Sec. 6.3.3: with the force correction, a field without mixed fourth
    derivatives then converges at fourth order).  tau_12 is Appendix C's (it
    zeroes C5, whose printed form is the scheme's); tau_22 solves C1 = 0 with
    the C1 of Appendix B (also the scheme's), which is linear in tau_22:
    12 theta (theta - nu) tau12 tau22 = 1 - theta^2
        - 12 (1 - theta^2)(1 - nu^2) (a3 E^2 + a2 tau12 E),
    a3 = (nu^2 - 2 theta nu + 1) / ((1 - theta^2)(1 - nu^2)^3),
    a2 = theta (nu - theta) / ((1 - theta^2)(1 - nu^2)^2), with E~ and nu from
    (lam, mu) by the 2D relations.  (Appendix C's printed tau_22 does not zero
    C1.)"""
    tau12, _ = fourth_order_taus(lam, mu, theta)
    nu = lam / (lam + 2.0 * mu)
    E = (lam + 2.0 * mu) * (1.0 - nu * nu)
    th = theta
    c, d = 1.0 - th * th, 1.0 - nu * nu
    a3 = (nu * nu - 2.0 * th * nu + 1.0) / (c * d ** 3)
    a2 = th * (nu - th) / (c * d ** 2)
    tau22 = (1.0 - th * th - 12.0 * c * d * (a3 * E * E + a2 * tau12 * E)) / (12.0 * th * (th - nu) * tau12)
    return tau12, tau22


# ----------------------------------------------------------------------------
# The pseudo-time step through the C oracle
# ----------------------------------------------------------------------------

def zero_state(nx: int, ny: int, q: int = 8) -> np.ndarray:
    """Initial populations at the equilibrium of u_0 = 0, i.e. all zero
    (Eq. init_cond with Table 1)."""
    return np.zeros((q, ny, nx), dtype=np.float64)


def run(f: np.ndarray, gx: np.ndarray, gy: np.ndarray, rates: np.ndarray,
        nsteps: int = 1) -> np.ndarray:
    """Advance pre-collision populations f[q, ny, nx] by ``nsteps`` pseudo-time
    steps (collision of Eq. collision at every node, then Eq. streaming);
    returns a new array."""
    q, ny, nx = f.shape
    fin = np.ascontiguousarray(f, dtype=np.float64)
    gx = np.ascontiguousarray(gx, dtype=np.float64)
    gy = np.ascontiguousarray(gy, dtype=np.float64)
    w = np.ascontiguousarray(rates, dtype=np.float64)
    assert gx.shape == (ny, nx) and gy.shape == (ny, nx) and w.shape == (7,)
    out = np.empty_like(fin)
    tmp = np.empty_like(fin)
    rc = _load().oracle_run(nx, ny, q, _ptr(fin), _ptr(gx), _ptr(gy), _ptr(w), int(nsteps),
                            _ptr(out), _ptr(tmp))
    if rc != 0:
        raise ValueError("oracle_run rejected its arguments")
    return out


def collide(f: np.ndarray, gx: np.ndarray, gy: np.ndarray, rates: np.ndarray) -> np.ndarray:
    """Post-collision populations f* (the per-node collision map only)."""
    q, ny, nx = f.shape
    fin = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(fin)
    rc = _load().oracle_collide(nx, ny, q, _ptr(fin), _ptr(np.ascontiguousarray(gx, np.float64)),
                                _ptr(np.ascontiguousarray(gy, np.float64)),
                                _ptr(np.ascontiguousarray(rates, np.float64)), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_collide rejected its arguments")
    return out


def moments(f: np.ndarray) -> np.ndarray:
    """Collision-basis moments [m_10, m_01, m_11, m_s, m_d, m_12, m_21, m_22(, m_00)]."""
    q, ny, nx = f.shape
    fin = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(fin)
    if _load().oracle_moments(nx, ny, q, _ptr(fin), _ptr(out)) != 0:
        raise ValueError("oracle_moments rejected its arguments")
    return out


def fields(f: np.ndarray, gx: np.ndarray, gy: np.ndarray, rates: np.ndarray) -> np.ndarray:
    """Solution fields [u_x, u_y, sigma_xx, sigma_yy, sigma_xy] (lattice units)
    of the pre-collision state f (Table 2, Eq. compute_bared)."""
    q, ny, nx = f.shape
    fin = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty((5, ny, nx), dtype=np.float64)
    rc = _load().oracle_fields(nx, ny, q, _ptr(fin), _ptr(np.ascontiguousarray(gx, np.float64)),
                               _ptr(np.ascontiguousarray(gy, np.float64)),
                               _ptr(np.ascontiguousarray(rates, np.float64)), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_fields rejected its arguments")
    return out


def raw_moment_inverse(q: int = 8) -> np.ndarray:
    out = np.empty((q, q), dtype=np.float64)
    if _load().oracle_raw_moment_inverse(q, _ptr(out)) != 0:
        raise ValueError("bad q")
    return out


# ----------------------------------------------------------------------------
# Pseudo-time iteration to steady state (Sec. 2.1) and grid norms (Sec. 6.1)
# ----------------------------------------------------------------------------

def residual(u_now: np.ndarray, u_prev: np.ndarray, k: int) -> tuple[float, float]:
    """Steady-state residual over a window of k steps.

    The paper stops when the time derivative of u is below a tolerance "in
    some norm" (Sec. 2.1).  Reading: r_inf = max|u^n - u^{n-k}| /
    (k * max|u^n|) with max over nodes and components, and the L2 analogue
    r_2 = ||u^n - u^{n-k}||_2 / (k * ||u^n||_2); r = 0 when u^n = 0.
    """
    d = u_now - u_prev
    umax = float(np.max(np.abs(u_now))) if u_now.size else 0.0
    u2 = float(np.sqrt(np.sum(u_now * u_now)))
    dmax = float(np.max(np.abs(d))) if d.size else 0.0
    d2 = float(np.sqrt(np.sum(d * d)))
    r_inf = 0.0 if umax == 0.0 else dmax / (k * umax)
    r_2 = 0.0 if u2 == 0.0 else d2 / (k * u2)
    return r_inf, r_2


def solve(gx: np.ndarray, gy: np.ndarray, rates: np.ndarray, tol: float,
          check_every: int = 100, max_iters: int = 10_000_000, q: int = 8,
          f0: np.ndarray | None = None):
    """Iterate the pseudo-time step from the zero state until the residual
    (``residual``) drops below ``tol``.  Returns (f, iters, r_inf)."""
    ny, nx = gx.shape
    f = zero_state(nx, ny, q) if f0 is None else f0
    u_prev = fields(f, gx, gy, rates)[:2]
    it = 0
    r = float("inf")
    while it < max_iters:
        f = run(f, gx, gy, rates, check_every)
        it += check_every
        u = fields(f, gx, gy, rates)[:2]
        r, _ = residual(u, u_prev, check_every)
        if not np.all(np.isfinite(u)):
            raise FloatingPointError("oracle diverged at step %d" % it)
        if r < tol:
            break
        u_prev = u
    return f, it, r


def grid_norms(err: np.ndarray, dx: float) -> tuple[float, float]:
    """L2 and Linf grid norms of a vector field err[c, ny, nx] (Sec. 6.1):
    L2 = (dx^2 sum_i |e_i|_2^2)^(1/2), Linf = max_i |e_i|_inf."""
    l2 = float(np.sqrt(dx * dx * np.sum(err * err)))
    linf = float(np.max(np.abs(err)))
    return l2, linf


# ----------------------------------------------------------------------------
# Leading-order error constants (Sec. 4, Appendix B) and the force correction
# ----------------------------------------------------------------------------

def error_constants_printed(E: float, nu: float, theta: float = THETA_STANDARD,
                            tau12: float = 0.5, tau21: float | None = None,
                            tau22: float = 0.5) -> np.ndarray:
    """[C1..C5, D1..D3] exactly as printed in Appendix B (functions of the
    dimensionless Young's modulus E, Poisson's ratio nu, theta and the
    higher-order relaxation times).  See ``leading_error_axis`` for how they
    compare with the scheme's exact discrete leading error."""
    th, t12, t22 = theta, tau12, tau22
    t21 = tau12 if tau21 is None else tau21
    c, d = 1.0 - th * th, 1.0 - nu * nu
    q = th * th * (1.0 + nu) + nu - 2.0 * th - 1.0
    C1 = ((nu ** 2 - 2 * th * nu + 1) / (c * d ** 3) * E ** 3
          + th * (nu - th) * t12 / (c * d ** 2) * E ** 2
          + (-1 + th ** 2 + 12 * th * (th - nu) * t12 * t22) / (12 * c * d) * E)
    C2 = (((1 - nu) ** 3 + 4 * th * (nu ** 3 - nu ** 2 + 3 * nu + 1)
           + th ** 2 * (5 * nu ** 3 - 15 * nu ** 2 - nu - 5)) / (8 * c * d ** 3) * E ** 3
          + (2 * th * ((1 - nu) * nu + th ** 2 * (1 + nu) - th * (1 + nu ** 2)) * t12
             + (1 - th) * (1 - nu) * (1 + 2 * th - nu - th ** 2 * (1 + nu)) * t21)
          / (-4 * th * c * d ** 2) * E ** 2
          + ((2 * th ** 2 - 3 * th + 1) * (1 + 3 * th * (1 - nu) - 5 * nu)
             + 24 * th * (th - nu) * t12 * t22) / (24 * c * d) * E)
    C3 = (((1 - nu) ** 2 * (3 + nu) + 4 * th * (-nu ** 3 + 3 * nu ** 2 + nu + 1)
           - th ** 2 * (5 * nu ** 3 - 3 * nu ** 2 + 7 * nu + 7)) / (8 * th * c * d ** 3) * E ** 3
          + (-2 * (1 - th) * th * (nu - 2 * th - 1) * (1 - nu) * t12
             - ((1 + th) * (1 - nu) ** 2 + th ** 3 * (1 + nu) ** 2 + th ** 2 * (nu ** 2 - 2 * nu - 3))
             * t21) / (4 * th * c * d ** 2) * E ** 2
          + ((1 - th) * (1 - nu - th * (1 + nu) - 2 * th ** 2 * (2 + nu))
             - 4 * c * (1 - nu) * t12 * t22 + 4 * q * t21 * t22) / (8 * c * d) * E
          + th * t22 / 4)
    C4 = ((16 * th * nu + (1 - nu) ** 2 * (3 + nu) - th ** 2 * (nu ** 3 + 9 * nu ** 2 - 5 * nu + 11))
          / (8 * th * c * d ** 3) * E ** 3
          + (c * (1 - nu) * (th * nu + nu + th - 1) * t12 - 2 * th * q * t21)
          / (4 * th * c * d ** 2) * E ** 2
          + (c * (2 * (2 - nu) - 3 * th * (5 + nu)) - 12 * c * (1 - nu) * t12 * t22
             + 12 * q * t21 * t22) / (24 * c * d) * E
          + th * t22 / 4)
    C5 = (E ** 3 / (8 * th * (1 + nu) ** 3) - (1 - th) * t12 / (4 * th * (1 + nu) ** 2) * E ** 2
          - (3 * th - 2) / (24 * (1 + nu)) * E)
    D1 = ((nu ** 2 - 2 * th * nu + 1) / (c * d ** 2) * E ** 2
          + th * (nu - th) * t12 / (c * d ** 2) * E - 0.25)
    D2 = (((1 - nu) ** 2 + 8 * th * nu - th ** 2 * (5 * nu ** 2 - 2 * nu + 5)) / (4 * th * c * d ** 2) * E ** 2
          - q * t21 / (2 * c * d ** 2) * E - th / 2)
    D3 = E ** 2 / (4 * th * (1 + nu) ** 2) + t12 / (2 * (1 + nu)) * E - th / 4
    return np.array([C1, C2, C3, C4, C5, D1, D2, D3])


def error_constants_read(E: float, nu: float, theta: float = THETA_STANDARD,
                         tau12: float = 0.5, tau21: float | None = None,
                         tau22: float = 0.5) -> np.ndarray:
    """[C1..C5, D1..D3] of Appendix B with the readings of three misprints
    applied (the scheme's exact discrete leading error, ``leading_error_exact``,
    decides them):

    * C2: the E^3 term is divided by 8 theta (1 - theta^2)(1 - nu^2)^3, like the
      E^3 terms of C3 and C4 (printed: 8 (1 - theta^2)(1 - nu^2)^3);
    * D1: the E term is theta (nu - theta) tau12 E / ((1 - theta^2)(1 - nu^2))
      (printed: (1 - nu^2)^2 in the denominator);
    * D2: the E term is -q tau21 E / (2 (1 - theta^2)(1 - nu^2)) with
      q = theta^2 (1 + nu) + nu - 2 theta - 1 (printed: (1 - nu^2)^2).

    The other five constants are the printed ones."""
    th = theta
    t21 = tau12 if tau21 is None else tau21
    c, d = 1.0 - th * th, 1.0 - nu * nu
    q = th * th * (1.0 + nu) + nu - 2.0 * th - 1.0
    out = error_constants_printed(E, nu, theta=theta, tau12=tau12, tau21=tau21, tau22=tau22).copy()
    p2 = ((1 - nu) ** 3 + 4 * th * (nu ** 3 - nu ** 2 + 3 * nu + 1)
          + th ** 2 * (5 * nu ** 3 - 15 * nu ** 2 - nu - 5))
    out[1] += p2 * E ** 3 * (1.0 / (8 * th * c * d ** 3) - 1.0 / (8 * c * d ** 3))
    out[5] += th * (nu - th) * tau12 * E * (1.0 / (c * d) - 1.0 / (c * d ** 2))
    out[6] += -q * t21 * E * (1.0 / (2 * c * d) - 1.0 / (2 * c * d ** 2))
    return out


def leading_error_exact(E: float, nu: float, theta: float = THETA_STANDARD,
                        tau12: float = 0.5, tau22: float = 0.5,
                        ks: tuple[float, float] = (0.01, 0.02)) -> tuple[np.ndarray, dict]:
    """[C1..C5, D1..D3] of the scheme itself, from its exact one-step operator
    (``fourier.amplification_matrix``), in the sign convention of Appendix B.

    Eq. ux_order2 (and its y twin) says that the displacement of a plane wave
    u = U exp(i k.x), k = kappa (c, s), obeys to O(kappa^4)
        d/dt U = (-M(k) + sigma A(k)) U + (1 - sigma Dm(k)) g_hat,
    with M the Navier-Cauchy symbol (mu kappa^2 + K k k^T), A the symbol of the
    C-terms (A_xx = C1 c^4 + C3 c^2 s^2 + C5 s^4, A_xy = C2 c^3 s + C4 c s^3,
    A_yx = C2 c s^3 + C4 c^3 s, A_yy = C1 s^4 + C3 c^2 s^2 + C5 c^4, times
    kappa^4), Dm that of the D-terms, and sigma = -1 (the sign reading of the
    printed constants).  Per time step (lattice units):

    * free decay (g = 0): the two slow eigenvalues of the one-step operator
      have log lambda = -s_j kappa^2 + sigma l_j kappa^4 with
      l_L = C1 (c^6 + s^6) + (C2 + C3 + C4 + C5) c^2 s^2 and
      l_T = C5 (c^6 + s^6) + (C1 + C3 - C2 - C4) c^2 s^2 (first-order
      perturbation of the symmetric M): c = 1 gives C1 and C5, c = s gives C3
      and C2 + C4;
    * the displacement of the slow eigenvectors tilts from k (resp. k-perp)
      by sigma kappa^2 cs (c^2 - s^2)(C5 - C1 + C4) / (-K) (longitudinal) and
      sigma kappa^2 cs (c^2 - s^2)(C5 - C1 + C2) / K (transverse): at
      tan(phi) = 1/2 these give C4 and C2 separately;
    * steady state for g = M U0: U - U0 = sigma M^-1 (A - Dm M) U0, whose
      entries give E1 = C1 - (mu + K) D1, E5 = C5 - mu D3,
      E2 = C2 - K D1 - mu D2 and, as checks, E3 = C3 - mu D1 - (mu + K) D3 - K D2
      and E4 = C4 - K D3 - (mu + K) D2.

    Each coefficient is extrapolated to kappa -> 0 from kappa = ks (Richardson
    in kappa^2).  The dict holds the three over-determined checks (C2 + C4
    from the eigenvalues minus the sum from the tilts, and the residuals of
    the E3 and E4 relations), which vanish when the structure of Eq. ux_order2
    holds."""
    from . import fourier as F
    lam, mu = lame_2d(E, nu)
    K = lam + mu
    rates = relaxation_rates(lam, mu, theta=theta, tau12=tau12, tau22=tau22)
    Mm = F.moment_matrix()

    def extrapolate(f):
        a, b = f(ks[0]), f(ks[1])
        return (4.0 * a - b) / 3.0

    def slow_modes(phi, kappa):
        cph, sph = np.cos(phi), np.sin(phi)
        vL, vT = np.array([cph, sph]), np.array([-sph, cph])
        w, V = np.linalg.eig(F.amplification_matrix(rates, kappa * cph, kappa * sph))
        out = {}
        for j in np.argsort(-np.abs(w))[:2]:
            U = Mm[:2] @ V[:, j]
            kind = "L" if abs(np.vdot(vL, U)) > abs(np.vdot(vT, U)) else "T"
            own, other = (vL, vT) if kind == "L" else (vT, vL)
            out[kind] = (float(np.log(w[j]).real), float((np.vdot(other, U) / np.vdot(own, U)).real))
        return out

    def rate(phi, kind):
        s2 = (mu + K) if kind == "L" else mu
        return extrapolate(lambda kap: (slow_modes(phi, kap)[kind][0] + s2 * kap * kap) / kap ** 4)

    def tilt(phi, kind):
        return extrapolate(lambda kap: slow_modes(phi, kap)[kind][1] / kap ** 2)

    sigma = -1.0
    C1, C5 = sigma * rate(0.0, "L"), sigma * rate(0.0, "T")
    SL, ST = 4.0 * sigma * rate(np.pi / 4, "L"), 4.0 * sigma * rate(np.pi / 4, "T")
    C3 = (SL + ST) / 2.0 - C1 - C5
    phi = np.arctan(0.5)
    g = np.cos(phi) * np.sin(phi) * (np.cos(phi) ** 2 - np.sin(phi) ** 2)    # = 0.24
    C4 = sigma * tilt(phi, "L") * (-K) / g - C5 + C1
    C2 = sigma * tilt(phi, "T") * K / g - C5 + C1

    A = F.operator(rates)
    Bx, By = F.force_vectors(rates)

    def steady_Q(ph, kappa):
        cph, sph = np.cos(ph), np.sin(ph)
        kx, ky = kappa * cph, kappa * sph
        Mk = np.array([[mu * kappa ** 2 + K * kx * kx, K * kx * ky],
                       [K * kx * ky, mu * kappa ** 2 + K * ky * ky]])
        S = F.shift_diag(kx, ky)
        cols = []
        for U0 in (np.array([1.0, 0.0]), np.array([0.0, 1.0])):
            gh = Mk @ U0
            fh = np.linalg.solve(np.eye(8) - S[:, None] * A, S * (Bx * gh[0] + By * gh[1]))
            U = Mm[:2] @ fh + 0.5 * gh              # u = m_10 + g/2 (Table 2)
            cols.append(sigma * (Mk @ (U - U0)).real / kappa ** 4)
        return np.stack(cols, axis=1)

    Q0 = extrapolate(lambda kap: steady_Q(0.0, kap))
    Qp = extrapolate(lambda kap: steady_Q(phi, kap))
    E1, E5 = Q0[0, 0], Q0[1, 1]
    cph, sph = np.cos(phi), np.sin(phi)
    E3 = (Qp[0, 0] - E1 * cph ** 4 - E5 * sph ** 4) / (cph * cph * sph * sph)
    E2, E4 = np.linalg.solve(np.array([[cph ** 3 * sph, cph * sph ** 3], [cph * sph ** 3, cph ** 3 * sph]]),
                             np.array([Qp[0, 1], Qp[1, 0]]))
    D1 = (C1 - E1) / (mu + K)
    D3 = (C5 - E5) / mu
    D2 = (C2 - K * D1 - E2) / mu
    checks = {"C2+C4": (SL - ST) / 2.0 - (C2 + C4),
              "E3": C3 - mu * D1 - (mu + K) * D3 - K * D2 - E3,
              "E4": C4 - K * D3 - (mu + K) * D2 - E4}
    return np.array([C1, C2, C3, C4, C5, D1, D2, D3]), checks


def corrected_force_fd(gx: np.ndarray, gy: np.ndarray, D) -> tuple[np.ndarray, np.ndarray]:
    """Force with the higher-order correction of Eqs. force_correction_x/y in
    lattice units, g' = g - (D1 dxx gx + D2 dxy gy + D3 dyy gx) (y analogous),
    derivatives by periodic central differences on the lattice."""
    D1, D2, D3 = D

    def dxx(a):
        return np.roll(a, -1, axis=1) - 2.0 * a + np.roll(a, 1, axis=1)

    def dyy(a):
        return np.roll(a, -1, axis=0) - 2.0 * a + np.roll(a, 1, axis=0)

    def dxy(a):
        return 0.25 * (np.roll(a, (-1, -1), axis=(0, 1)) - np.roll(a, (1, -1), axis=(0, 1))
                       - np.roll(a, (-1, 1), axis=(0, 1)) + np.roll(a, (1, 1), axis=(0, 1)))

    gxc = gx - (D1 * dxx(gx) + D2 * dxy(gy) + D3 * dyy(gx))
    gyc = gy - (D3 * dxx(gy) + D2 * dxy(gx) + D1 * dyy(gy))
    return np.ascontiguousarray(gxc), np.ascontiguousarray(gyc)


def leading_error_axis(E: float, nu: float, tau12: float = 0.5, tau22: float = 0.5,
                       theta: float = THETA_STANDARD, n: int = 2048) -> tuple[float, float]:
    """Exact-discrete leading-order error coefficients of axis-aligned modes.

    For a displacement plane wave along x (k = 2 pi / L), the scheme's steady
    state (per-mode closed form, ``fourier.steady_state_modes``) differs from
    the exact solution by eps^2 u2 + O(eps^4); writing the error source of
    Eq. ux_order2 as A k^4 u for such a mode, the longitudinal wave (u along
    k) gives A1 = (mu + K) u2 / k^2 and the transverse one A5 = mu u2 / k^2.
    In the notation of Appendix B, A1 corresponds to -(C1 - (mu + K) D1) and A5
    to -(C5 - mu D3) (the printed error equation carries the opposite sign)."""
    from . import fourier as F
    lam, mu = lame_2d(E, nu)
    K = lam + mu
    rates = relaxation_rates(lam, mu, theta=theta, tau12=tau12, tau22=tau22)
    k = 2.0 * np.pi
    out = []
    for Ux, Uy, modulus in ((1.0, 0.0, mu + K), (0.0, 1.0, mu)):
        # force of u = (Ux, Uy) cos(k x): b = mu k^2 U + K k (k . U)
        k1 = k / n
        bx = mu * k1 * k1 * Ux + K * k1 * k1 * Ux
        by = mu * k1 * k1 * Uy
        ks, fh, flh = F.steady_state_modes(n, n, [(1, 0, bx, by)], rates)
        u = flh[0, 0] if Ux else flh[0, 1]
        u2 = float(np.real(u - 1.0)) * n * n
        out.append(modulus * u2 / (k * k))
    return out[0], out[1]
