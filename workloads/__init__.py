"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the lattice Boltzmann scheme itself.  It
produces body-force fields (and, for manufactured solutions, the exact
displacement and stress of the target PDE), material parameters, and the
problem lists of the batched and served workloads.  Both the CUDA library and
the oracle consume what it returns; it imports neither.

Conventions (lattice units, Delta x = Delta t = 1):
  * node (n_x, n_y), 0 <= n < N, sits at x = n + 1/2 (the lattice is offset by
    half a spacing from the periodic domain edge, Sec. 5.1 of the paper);
  * a plane wave on an nx-by-ny lattice has integer wave numbers (kx, ky) and
    wave vector k = 2 pi (kx / nx, ky / ny);
  * the Lame parameters are the lattice-unit moduli lambda~, mu~ of the
    paper's Sec. 2.2; with a dimensionless Young's modulus E~ they follow the
    2D relations lambda = E nu / (1 - nu^2), mu = E / (2 (1 + nu))
    (Eq. material_relations);
  * a manufactured displacement u^ gives the lattice body force
    g = -mu lap(u^) - K grad(div u^), K = lambda + mu (Eq. manu_eq with a
    time-independent solution; the paper's forcing g = eps^2 g^(2) with
    derivatives taken per node spacing), and the lattice stress
    sigma = K div(u) I + mu (grad u + grad u^T - div(u) I) (Eq. stress),
    which is the paper's dimensionless stress times eps = 1/N.

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014), implemented
here from its published definition, so every platform draws the same values.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 counter-based generator: state += golden gamma, then the
    variant-13 finaliser of MurmurHash3."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniform_open(self) -> float:
        """Uniform in (0, 1]."""
        return ((self.next_u64() >> 11) + 1) * (1.0 / (1 << 53))

    def normal(self) -> float:
        """Standard normal by the Box-Muller transform."""
        u1 = self.uniform_open()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] (modulo bias below 2^-50 for small ranges)."""
        return lo + self.next_u64() % (hi - lo + 1)


def lame_2d(E: float, nu: float) -> tuple[float, float]:
    """(lambda, mu) of the 2D medium, Eq. material_relations."""
    return E * nu / (1.0 - nu * nu), E / (2.0 * (1.0 + nu))


# ----------------------------------------------------------------------------
# Plane-wave fields
# ----------------------------------------------------------------------------

@dataclass
class PlaneWaves:
    """A real vector field Re sum_m (ax_m, ay_m) exp(i (k1_m x + k2_m y)) on an
    nx-by-ny lattice; (kx_m, ky_m) are integer wave numbers."""
    nx: int
    ny: int
    kx: np.ndarray   # int, (M,)
    ky: np.ndarray   # int, (M,)
    ax: np.ndarray   # complex, (M,)
    ay: np.ndarray   # complex, (M,)

    @property
    def k1(self) -> np.ndarray:
        return 2.0 * np.pi * self.kx / self.nx

    @property
    def k2(self) -> np.ndarray:
        return 2.0 * np.pi * self.ky / self.ny

    def modes(self):
        """(kx, ky, ax, ay) tuples."""
        return list(zip(self.kx.tolist(), self.ky.tolist(), self.ax.tolist(), self.ay.tolist()))

    def grid(self, amps: np.ndarray | None = None) -> np.ndarray:
        """Evaluate Re sum_m amps_m exp(i k_m.x) at every node, (ny, nx) float64.
        Separable: one real matrix product [cos(k2 y), sin(k2 y)] @ [P; Q]."""
        if amps is None:
            raise ValueError("amps required")
        x = np.arange(self.nx, dtype=np.float64) + 0.5
        y = np.arange(self.ny, dtype=np.float64) + 0.5
        ex = np.exp(1j * np.outer(self.k1, x)) * amps[:, None]      # (M, nx)
        cy = np.cos(np.outer(y, self.k2))                            # (ny, M)
        sy = np.sin(np.outer(y, self.k2))
        left = np.concatenate([cy, sy], axis=1)                      # (ny, 2M)
        right = np.concatenate([ex.real, -ex.imag], axis=0)          # (2M, nx)
        return np.ascontiguousarray(left @ right)

    def at(self, amps: np.ndarray, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        """Evaluate at arbitrary positions (lattice units)."""
        out = np.zeros(np.broadcast(X, Y).shape)
        for k1, k2, a in zip(self.k1, self.k2, amps):
            out += np.real(a * np.exp(1j * (k1 * X + k2 * Y)))
        return out


@dataclass
class Manufactured:
    """A manufactured periodic solution: displacement plane waves, the matching
    lattice body force, and the exact lattice stress."""
    lam: float
    mu: float
    u: PlaneWaves                     # displacement amplitudes in (ax, ay)
    fx: np.ndarray = field(init=False)  # force amplitudes, per mode
    fy: np.ndarray = field(init=False)
    sxx: np.ndarray = field(init=False)
    syy: np.ndarray = field(init=False)
    sxy: np.ndarray = field(init=False)

    def __post_init__(self):
        k1, k2 = self.u.k1, self.u.k2
        Ux, Uy = self.u.ax, self.u.ay
        K = self.lam + self.mu
        kk = k1 * k1 + k2 * k2
        kdotU = k1 * Ux + k2 * Uy
        # b = -mu lap u - K grad div u; lap -> -|k|^2, grad div -> -k (k.U)
        self.fx = self.mu * kk * Ux + K * k1 * kdotU
        self.fy = self.mu * kk * Uy + K * k2 * kdotU
        div = 1j * kdotU
        self.sxx = K * div + self.mu * (2j * k1 * Ux - div)
        self.syy = K * div + self.mu * (2j * k2 * Uy - div)
        self.sxy = self.mu * 1j * (k1 * Uy + k2 * Ux)

    def force(self) -> tuple[np.ndarray, np.ndarray]:
        return self.u.grid(self.fx), self.u.grid(self.fy)

    def force_modes(self):
        return list(zip(self.u.kx.tolist(), self.u.ky.tolist(), self.fx.tolist(), self.fy.tolist()))

    def exact(self) -> np.ndarray:
        """[u_x, u_y, sigma_xx, sigma_yy, sigma_xy] on the grid, (5, ny, nx)."""
        return np.stack([self.u.grid(a) for a in
                         (self.u.ax, self.u.ay, self.sxx, self.syy, self.sxy)])


def _pw(nx, ny, modes) -> PlaneWaves:
    kx = np.array([m[0] for m in modes], dtype=np.int64)
    ky = np.array([m[1] for m in modes], dtype=np.int64)
    ax = np.array([m[2] for m in modes], dtype=np.complex128)
    ay = np.array([m[3] for m in modes], dtype=np.complex128)
    return PlaneWaves(nx, ny, kx, ky, ax, ay)


def sinusoid(n: int, k: int, lam: float, mu: float, ny: int | None = None) -> Manufactured:
    """The sweep field u_x = sin(2 pi k x~) cos(2 pi k y~), u_y = cos(2 pi k x~)
    sin(2 pi k y~) on the unit square sampled by an n-by-n lattice (curl free;
    its force is 2 a^2 (mu + K) u with a = 2 pi k / n)."""
    ny = n if ny is None else ny
    # sin(ax)cos(ay) = Re[-i/2 e^{i(ax+ay)} - i/2 e^{i(ax-ay)}]
    # cos(ax)sin(ay) = Re[-i/2 e^{i(ax+ay)} + i/2 e^{i(ax-ay)}]
    modes = [(k, k, -0.5j, -0.5j), (k, -k, -0.5j, 0.5j)]
    return Manufactured(lam, mu, _pw(n, ny, modes))


def paper_field(n: int, lam: float, mu: float, A: float = 9e-4, B: float = 7e-4) -> Manufactured:
    """The field of the paper's first convergence study (Sec. 6.3.1):
    u_x = A cos(2 pi x~) sin(2 pi y~), u_y = B sin(2 pi x~) cos(2 pi y~)."""
    # cos(ax)sin(ay) = Re[-i/2 e^{i(+,+)} + i/2 e^{i(+,-)}]
    # sin(ax)cos(ay) = Re[-i/2 e^{i(+,+)} - i/2 e^{i(+,-)}]
    modes = [(1, 1, -0.5j * A, -0.5j * B), (1, -1, 0.5j * A, -0.5j * B)]
    return Manufactured(lam, mu, _pw(n, n, modes))


def fourth_order_field(n: int, lam: float, mu: float, A: float = 9e-4, B: float = 7e-4) -> Manufactured:
    """The field of the fourth-order special case (Sec. 6.3.3):
    u_x = A (cos 2 pi x~ + sin 2 pi y~), u_y = B (sin 2 pi x~ + cos 2 pi y~)."""
    modes = [(1, 0, A + 0j, -1j * B), (0, 1, -1j * A, B + 0j)]
    return Manufactured(lam, mu, _pw(n, n, modes))


GAUSS_SIGMA = (120.0 ** -0.5, 123.0 ** -0.5, 118.0 ** -0.5, 125.0 ** -0.5)  # Sec. 6.3.5 table


def gaussian_hill(n: int, lam: float, mu: float, amp: float = 1e-3, sigma=GAUSS_SIGMA):
    """The Gaussian-hill manufactured solution of Sec. 6.3.5 on the unit square
    sampled by an n-by-n lattice:
      u_x = amp exp(-(x~ - 1/2)^2 / s1^2) exp(-(y~ - 1/2)^2 / s2^2) - mean,
      u_y = amp exp(-(x~ - 1/2)^2 / s3^2) exp(-(y~ - 1/2)^2 / s4^2) - mean,
    the means being amp pi s_a s_b erf(1/(2 s_a)) erf(1/(2 s_b)).  The field is
    periodic only approximately (it is ~1e-13 amp at the domain edge); the
    lattice force g = (-mu lap u - K grad div u) / n^2 (unit-square derivatives,
    E~ = 1 scaling of the moduli) has its small grid mean removed so that the
    periodic problem has a steady state.  Returns (gx, gy, exact) with exact the
    fields (5, n, n) [u_x, u_y, sigma_xx, sigma_yy, sigma_xy] in lattice units."""
    from math import erf, pi, sqrt
    s1, s2, s3, s4 = sigma
    K = lam + mu
    t = (np.arange(n, dtype=np.float64) + 0.5) / n - 0.5
    X, Y = np.meshgrid(t, t)               # X varies along x (columns)

    def hill(sa, sb):
        G = amp * np.exp(-X * X / (sa * sa)) * np.exp(-Y * Y / (sb * sb))
        gx_ = -2.0 * X / (sa * sa) * G
        gy_ = -2.0 * Y / (sb * sb) * G
        gxx = (4.0 * X * X / sa ** 4 - 2.0 / (sa * sa)) * G
        gyy = (4.0 * Y * Y / sb ** 4 - 2.0 / (sb * sb)) * G
        gxy = 4.0 * X * Y / (sa * sa * sb * sb) * G
        mean = amp * pi * sa * sb * erf(1.0 / (2.0 * sa)) * erf(1.0 / (2.0 * sb))
        return G - mean, gx_, gy_, gxx, gyy, gxy

    ux, ux_x, ux_y, ux_xx, ux_yy, ux_xy = hill(s1, s2)
    uy, uy_x, uy_y, uy_xx, uy_yy, uy_xy = hill(s3, s4)
    bx = -mu * (ux_xx + ux_yy) - K * (ux_xx + uy_xy)
    by = -mu * (uy_xx + uy_yy) - K * (ux_xy + uy_yy)
    gx = bx / (n * n)
    gy = by / (n * n)
    gx -= gx.mean()
    gy -= gy.mean()
    div = ux_x + uy_y
    sxx = K * div + mu * (2.0 * ux_x - div)
    syy = K * div + mu * (2.0 * uy_y - div)
    sxy = mu * (ux_y + uy_x)
    exact = np.stack([ux, uy, sxx / n, syy / n, sxy / n])
    return np.ascontiguousarray(gx), np.ascontiguousarray(gy), exact


def random_force(nx: int, ny: int, n_modes: int, kmax: int, seed: int) -> PlaneWaves:
    """Body force made of ``n_modes`` random Fourier modes: integer wave numbers
    (kx, ky) uniform in [-kmax, kmax]^2 without (0, 0); per component amplitude
    N(0, 1) / |k|^2; phase uniform in [0, 2 pi).  On the unit square
    b = sum_m a_m cos(2 pi (kx x~ + ky y~) + phi_m); the lattice force is
    g = b / max(nx, ny)^2 (dimensionless Young's modulus 1).  Zero mean by
    construction.  Returned as plane waves whose (ax, ay) are the complex
    force amplitudes."""
    rng = SplitMix64(seed)
    scale = 1.0 / float(max(nx, ny)) ** 2
    modes = []
    while len(modes) < n_modes:
        kx = rng.randint(-kmax, kmax)
        ky = rng.randint(-kmax, kmax)
        if kx == 0 and ky == 0:
            continue
        k2 = float(kx * kx + ky * ky)
        ax = rng.normal() / k2
        ay = rng.normal() / k2
        phi = 2.0 * math.pi * rng.uniform()
        e = complex(math.cos(phi), math.sin(phi)) * scale
        modes.append((kx, ky, ax * e, ay * e))
    return _pw(nx, ny, modes)


def random_force_grid(pw: PlaneWaves) -> tuple[np.ndarray, np.ndarray]:
    return pw.grid(pw.ax), pw.grid(pw.ay)


# ----------------------------------------------------------------------------
# Batched and served workloads
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    """One periodic problem of the batched or served workload."""
    pid: int
    nx: int
    ny: int
    nu: float
    lam: float
    mu: float
    force: PlaneWaves
    dtype: str = "f32"
    arrival: float = 0.0   # seconds, served workload only


def log_uniform_side(rng: SplitMix64, lo: int, hi: int) -> int:
    return int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * rng.uniform())))


def batched_problems(count: int = 2048, lo: int = 32, hi: int = 1024, nu_max: float = 0.45,
                     n_modes: int = 8, kmax: int = 4, seed: int = 0x5EED_BA7C4ED,
                     E: float = 1.0) -> list[Problem]:
    """Independent periodic problems: nx, ny log-uniform in [lo, hi]
    (independently, so non-square), nu uniform in [0, nu_max], E~ = E,
    8-mode random body force (``random_force``)."""
    rng = SplitMix64(seed)
    out = []
    for pid in range(count):
        nx = log_uniform_side(rng, lo, hi)
        ny = log_uniform_side(rng, lo, hi)
        nu = nu_max * rng.uniform()
        lam, mu = lame_2d(E, nu)
        fseed = rng.next_u64()
        out.append(Problem(pid, nx, ny, nu, lam, mu, random_force(nx, ny, n_modes, kmax, fseed)))
    return out


def served_requests(count: int = 20000, rate_hz: float = 100.0, lo: int = 64, hi: int = 4096,
                    nu_max: float = 0.45, n_modes: int = 8, kmax: int = 4,
                    seed: int = 0x5E4FED, E: float = 1.0) -> list[Problem]:
    """Poisson-arrival solve requests: exponential inter-arrival times at
    ``rate_hz``; sides log-uniform in [lo, hi]; nu uniform in [0, nu_max];
    storage FP32 or FP16-shifted with probability 1/2 each."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for pid in range(count):
        t += -math.log(rng.uniform_open()) / rate_hz
        nx = log_uniform_side(rng, lo, hi)
        ny = log_uniform_side(rng, lo, hi)
        nu = nu_max * rng.uniform()
        lam, mu = lame_2d(E, nu)
        dtype = "f32" if rng.uniform() < 0.5 else "f16s"
        fseed = rng.next_u64()
        out.append(Problem(pid, nx, ny, nu, lam, mu, random_force(nx, ny, n_modes, kmax, fseed),
                           dtype=dtype, arrival=t))
    return out


def random_populations(q: int, nx: int, ny: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Random populations (q, ny, nx), uniform in [-scale, scale), for single-step
    parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(rng.uniform(-scale, scale, size=(q, ny, nx)))


def random_field(nx: int, ny: int, seed: int, scale: float = 1.0, zero_mean: bool = False) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.uniform(-scale, scale, size=(ny, nx))
    if zero_mean:
        a -= a.mean()
    return np.ascontiguousarray(a)
