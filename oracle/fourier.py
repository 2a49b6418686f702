"""Linear-operator view of the scheme: one-step operator, von Neumann spectral
radius and the exact discrete steady state, mode by mode.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

The scheme is linear and translation invariant (Sec. 4).  One step maps the
pre-collision populations f(x, t) to

    f_i(x + c_i, t + 1) = sum_l A_il f_l(x, t) + (B_x g_x + B_y g_y)_i(x)

with A = M^-1 Lambda M^eq + M^-1 (I - Lambda) M (Eq. lbmvector).  M is the
population-to-moment matrix built from the moment definition (Eq. moments and
Eq. replace_raw; printed in Sec. 4), Lambda = diag(0, 0, w_11, w_s, w_d,
w_12, w_21, w_22), and M^eq maps populations to the Table 1 equilibria
(m_12^eq = theta m_10, m_21^eq = theta m_01, all others zero).  The force
enters the post-collision first moments with weight 1 (Eqs. coll10 and
coll10post together) and, through m_12^eq = theta*mbar_10 with
mbar_10 = m_10 + g_x/2, the post-collision m_12 with weight w_12*theta/2; B is
M^-1 applied to those weights.

Reading of a misprint: the M^eq printed in Sec. 4 repeats the m_12 row
(theta*(0 0 0 0 1 -1 -1 1)) where Table 1 asks for theta times the m_10 row.
Table 1 is followed here; ``printed_meq=True`` gives the printed matrix for the
test that documents the difference (the printed one keeps the paper's declared
unstable point nu = -0.4, E = 0.082 of Sec. 6.3.5 stable, Table 1 does not).

A plane wave f(x) = a exp(i k.x) turns one step into L(k) a with
L_ij = exp(-i k.c_i) A_ij (Eq. eigen); the scheme is stable when the spectral
radius of L stays <= 1 over k (Sec. 4).  For a force made of plane waves the
steady state of the damped iteration solves, per wave vector k != 0,

    (I - S(k) A) f_hat = S(k) (B_x gx_hat + B_y gy_hat),  S = diag(exp(-i k.c_i)),

which is exact for the discrete scheme (no truncation), so it pins steady
states at lattice sizes where time stepping the C oracle would take hours.
"""
from __future__ import annotations

import numpy as np

# Velocity table, paper's one-index order (Table "map between one-index and
# two-index notations for the populations").
CX = np.array([1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)
CY = np.array([0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)


def moment_matrix() -> np.ndarray:
    """M with rows m_10, m_01, m_11, m_s, m_d, m_12, m_21, m_22 (moment table of
    Sec. 4), built from m_ab = sum_i cx_i^a cy_i^b f_i (Eq. moments) and
    m_s = m_20 + m_02, m_d = m_20 - m_02 (Eq. replace_raw)."""
    def raw(a, b):
        return CX ** a * CY ** b
    return np.stack([raw(1, 0), raw(0, 1), raw(1, 1), raw(2, 0) + raw(0, 2),
                     raw(2, 0) - raw(0, 2), raw(1, 2), raw(2, 1), raw(2, 2)])


def equilibrium_matrix(theta: float, printed_meq: bool = False) -> np.ndarray:
    """M^eq: populations -> equilibrium moments (Table 1 reading by default)."""
    M = moment_matrix()
    E = np.zeros((8, 8))
    E[0] = M[0]
    E[1] = M[1]
    if printed_meq:
        E[5] = theta * M[5]
        E[6] = theta * M[6]
    else:
        E[5] = theta * M[0]
        E[6] = theta * M[1]
    return E


def relaxation_matrix(rates: np.ndarray) -> np.ndarray:
    w11, ws, wd, w12, w21, w22 = rates[:6]
    return np.diag([0.0, 0.0, w11, ws, wd, w12, w21, w22])


def operator(rates: np.ndarray, printed_meq: bool = False) -> np.ndarray:
    """Collision operator A of Eq. lbmvector."""
    theta = float(rates[6])
    M = moment_matrix()
    Minv = np.linalg.inv(M)
    Lam = relaxation_matrix(rates)
    return Minv @ Lam @ equilibrium_matrix(theta, printed_meq) + Minv @ (np.eye(8) - Lam) @ M


def force_vectors(rates: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Injection of (g_x, g_y) into the post-collision populations."""
    theta, w12, w21 = float(rates[6]), float(rates[3]), float(rates[4])
    Minv = np.linalg.inv(moment_matrix())
    ex = np.zeros(8)
    ex[0] = 1.0
    ex[5] = w12 * theta / 2.0
    ey = np.zeros(8)
    ey[1] = 1.0
    ey[6] = w21 * theta / 2.0
    return Minv @ ex, Minv @ ey


def shift_diag(kx: float, ky: float) -> np.ndarray:
    """S(k) = diag(exp(-i k.c_i))."""
    return np.exp(-1j * (kx * CX + ky * CY))


def amplification_matrix(rates: np.ndarray, kx: float, ky: float,
                         printed_meq: bool = False) -> np.ndarray:
    """L(k) of Eq. eigen."""
    return shift_diag(kx, ky)[:, None] * operator(rates, printed_meq)


def spectral_radius(rates: np.ndarray, nk: int = 50, nphi: int = 5,
                    printed_meq: bool = False) -> float:
    """sup over sampled wave vectors of rho(L(k)); k = khat (cos phi, sin phi),
    khat in [0, pi] (nk points), phi in [0, pi/4] (nphi points) (Sec. 4)."""
    A = operator(rates, printed_meq)
    best = 0.0
    for phi in np.linspace(0.0, np.pi / 4.0, nphi):
        for kh in np.linspace(0.0, np.pi, nk):
            L = shift_diag(kh * np.cos(phi), kh * np.sin(phi))[:, None] * A
            best = max(best, float(np.max(np.abs(np.linalg.eigvals(L)))))
    return best


def _field_rows(rates: np.ndarray) -> np.ndarray:
    """Linear map from (f_hat[8], gx_hat, gy_hat) to the 5 solution fields
    u_x, u_y, sigma_xx, sigma_yy, sigma_xy (Table 2, Eq. compute_bared)."""
    w11, ws, wd = rates[:3]
    M = moment_matrix()
    R = np.zeros((5, 10))
    R[0, :8] = M[0]
    R[0, 8] = 0.5
    R[1, :8] = M[1]
    R[1, 9] = 0.5
    mb11 = (1.0 - w11 / 2.0) * M[2]
    mbs = (1.0 - ws / 2.0) * M[3]
    mbd = (1.0 - wd / 2.0) * M[4]
    R[2, :8] = -(mbs + mbd) / 2.0
    R[3, :8] = -(mbs - mbd) / 2.0
    R[4, :8] = -mb11
    return R


def steady_state_modes(nx: int, ny: int, modes, rates: np.ndarray):
    """Exact steady state for a force g(x) = Re sum_m (gx_m, gy_m) exp(i k_m.x),
    k_m = 2 pi (kx_m / nx, ky_m / ny) with integers (kx_m, ky_m) != (0, 0).

    ``modes``: iterable of (kx, ky, gx_hat, gy_hat) (complex amplitudes).
    Returns (kvecs[m, 2], f_hat[m, 8], field_hat[m, 5]) such that each field
    is Re sum_m field_hat[m] exp(i k_m.x) over node positions x.
    """
    A = operator(rates)
    Bx, By = force_vectors(rates)
    R = _field_rows(rates)
    ks, fs, fl = [], [], []
    for kx, ky, gxh, gyh in modes:
        if kx % nx == 0 and ky % ny == 0:
            raise ValueError("the (0, 0) mode has no steady state unless its force is zero")
        k1 = 2.0 * np.pi * kx / nx
        k2 = 2.0 * np.pi * ky / ny
        S = shift_diag(k1, k2)
        lhs = np.eye(8) - S[:, None] * A
        rhs = S * (Bx * gxh + By * gyh)
        fh = np.linalg.solve(lhs, rhs)
        ks.append((k1, k2))
        fs.append(fh)
        fl.append(R @ np.concatenate([fh, [gxh, gyh]]))
    return np.array(ks), np.array(fs), np.array(fl)


def evaluate_modes(kvecs: np.ndarray, amps: np.ndarray, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Re sum_m amps[m] exp(i (k_m,x X + k_m,y Y)) at positions (X, Y)."""
    out = np.zeros(np.broadcast(X, Y).shape, dtype=np.float64)
    for (k1, k2), a in zip(kvecs, amps):
        out += np.real(a * np.exp(1j * (k1 * X + k2 * Y)))
    return out


def steady_state_grid(gx: np.ndarray, gy: np.ndarray, rates: np.ndarray,
                      chunk: int = 65536) -> np.ndarray:
    """Exact steady-state pre-collision populations f[8, ny, nx] for an
    arbitrary zero-mean force on the grid (all discrete Fourier modes, with
    numpy's FFT as the transform)."""
    ny, nx = gx.shape
    gxh = np.fft.fft2(gx)
    gyh = np.fft.fft2(gy)
    scale = max(np.max(np.abs(gxh)), np.max(np.abs(gyh)), 1e-300)
    if abs(gxh[0, 0]) > 1e-10 * scale or abs(gyh[0, 0]) > 1e-10 * scale:
        raise ValueError("force must have zero mean (the mean of u is conserved, Sec. 6.2)")
    A = operator(rates)
    Bx, By = force_vectors(rates)
    k2 = 2.0 * np.pi * np.fft.fftfreq(ny)[:, None] * np.ones((1, nx))
    k1 = 2.0 * np.pi * np.fft.fftfreq(nx)[None, :] * np.ones((ny, 1))
    k1 = k1.ravel()
    k2 = k2.ravel()
    gxf = gxh.ravel()
    gyf = gyh.ravel()
    fh = np.zeros((8, nx * ny), dtype=np.complex128)
    idx = np.arange(1, nx * ny)  # skip the (0, 0) bin: zero mean stays zero
    for s in range(0, idx.size, chunk):
        sel = idx[s:s + chunk]
        S = np.exp(-1j * (k1[sel, None] * CX[None, :] + k2[sel, None] * CY[None, :]))
        lhs = np.eye(8)[None] - S[:, :, None] * A[None]
        rhs = S * (Bx[None] * gxf[sel, None] + By[None] * gyf[sel, None])
        fh[:, sel] = np.linalg.solve(lhs, rhs[..., None])[..., 0].T
    f = np.real(np.fft.ifft2(fh.reshape(8, ny, nx), axes=(1, 2)))
    return np.ascontiguousarray(f)
