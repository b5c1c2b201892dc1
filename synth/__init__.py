"""Seeded synthetic inputs for the TDSE workloads.

This module only *samples the problem data* -- the initial wavefunction u0,
the static potential profile V0 and its time factor f(t) (so that
V(x, t) = f(t) V0(x)) or a general V(x, t), and the parameters of the
vector-potential pulse A(t)
-- on the spatial grid that the problem statement fixes.  It contains none of
the solver's arithmetic (no transforms, no phases, no quadrature, no phi = int
A); both the CPU oracle and the CUDA path receive exactly these arrays.

Grids (problem definition):
  * periodic, Sec. 2.1: x_j = -pi + 2 pi j / M, j = 0..M-1 on [-pi, pi]^d;
  * free space, Sec. 3.3: x_j = -1 + 2 (j-1) / M, j = 1..M on [-1, 1]^d.

Workloads (shapes/values follow the paper's 1D/2D examples, Sec. 7):
  * ``periodic_1d_cosine``  -- 1D periodic, N=128, Gaussian packet, 4-mode
    cosine potential with time factor 1 + 0.5 sin 2t, A = 0, T=1, dt=1e-2;
  * ``periodic_2d_wells``   -- 2D periodic 512^2, three Gaussians, four
    attractive Gaussian wells, pulse A(t) = 2 sin^2(pi t/2) sin(10 t) (1,0),
    T=2, dt=1e-3;
  * ``periodic_1d_batch_member`` -- one member of the uneven 1D batch
    (N in {256..16384}), T=1, dt=1e-3;
  * ``moving_well_1d`` -- Example 1: moving periodic Gaussian well
    (V0 = 300, beta = 0.2, speed c, T = 2 pi / 15), u0 its ground state
    (Fourier-Galerkin eigensolve of the static well); ``moving_wells_2d``,
    ``free_moving_wells`` -- drifting wells (non-separable V(x, t));
  * ``free_bump_gaussians`` -- free space on [-1,1]^d (default 256^2):
    Gaussians (sigma ~ U[0.08,0.15], centres ~ U[-0.4,0.4]^d) times the
    C-infinity window exp(1 - 1/(1 - r^2)), r = |x| / 0.95, for u0 and for
    four attractive wells of depth U[5,20]; pulse A0 = 2, omega = 10 along
    (1,0), T = 1, dt = 5e-4.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional, Sequence

import numpy as np

PERIODIC = 0
FREE = 1


def periodic_grid(M: int) -> np.ndarray:
    """x_j = -pi + 2 pi j / M, j = 0..M-1 (Sec. 2.1)."""
    return -math.pi + 2.0 * math.pi * np.arange(M, dtype=np.float64) / M


def free_grid(M: int) -> np.ndarray:
    """x_j = -1 + 2 (j-1) / M, j = 1..M (Sec. 3.3)."""
    return -1.0 + 2.0 * np.arange(M, dtype=np.float64) / M


@dataclasses.dataclass(frozen=True)
class Pulse:
    """A(t) = A0 sin^2(pi t / T_pulse) sin(omega t) * direction.

    The workload tables use sin(omega t); the paper's eq. (apulse) prints
    cos(omega t).  Only the sampling of A is defined here.
    """

    A0: float
    omega: float
    T_pulse: float
    direction: tuple

    def A(self, t) -> np.ndarray:
        t = np.asarray(t, dtype=np.float64)
        amp = self.A0 * np.sin(math.pi * t / self.T_pulse) ** 2 * np.sin(self.omega * t)
        return np.multiply.outer(amp, np.asarray(self.direction, dtype=np.float64))


@dataclasses.dataclass
class Instance:
    """One TDSE problem: data on the grid plus time stepping parameters."""

    bc: int
    shape: tuple
    u0: np.ndarray            # complex128, shape `shape`
    V0: np.ndarray            # float64, shape `shape` (V(x, 0) when Vt is set)
    vfac: Callable            # f(t), vectorised; V(x,t) = f(t) V0(x)
    pulse: Optional[Pulse]    # None means A = 0
    dt: float
    nsteps: int
    name: str = ""
    Vt: Optional[Callable] = None   # general V: t -> V(x, t) on the grid (vfac unused)

    @property
    def dim(self) -> int:
        return len(self.shape)

    @property
    def t_max(self) -> float:
        return self.nsteps * self.dt

    def vfac_table(self, sub: int = 8) -> np.ndarray:
        """f(t) sampled at t = m dt / sub, m = 0 .. sub*nsteps."""
        m = np.arange(sub * self.nsteps + 1, dtype=np.float64)
        return np.asarray(self.vfac(m * self.dt / sub), dtype=np.float64).reshape(-1)

    def V_at(self, t: float) -> np.ndarray:
        """V(x, t) on the grid."""
        if self.Vt is not None:
            return np.asarray(self.Vt(t), dtype=np.float64)
        return float(np.asarray(self.vfac(t)).reshape(-1)[0]) * self.V0

    def potential_table(self, times) -> np.ndarray:
        """V(x, t) on the grid at each of `times`: array [len(times)] + shape."""
        return np.stack([self.V_at(float(t)) for t in times]).astype(np.float64)


def _const_one(t):
    return np.ones_like(np.asarray(t, dtype=np.float64))


def _grid_norm(u: np.ndarray, h: float) -> float:
    return math.sqrt(float(np.sum(np.abs(u) ** 2)) * h ** u.ndim)


def _periodised_gaussian_2d(X, Y, cx, cy, sigma, images=3):
    """sum over the lattice images |m| <= images of exp(-|x - c - 2 pi m|^2 / (2 sigma^2))
    on the grid X, Y (meshgrid, indexing "ij"): the Gaussian and the image
    sum factor into the product of two 1D image sums along the grid lines."""
    L = 2.0 * math.pi
    x, y = X[:, 0], Y[0, :]
    gx = sum(np.exp(-(x - cx - L * m) ** 2 / (2.0 * sigma * sigma)) for m in range(-images, images + 1))
    gy = sum(np.exp(-(y - cy - L * m) ** 2 / (2.0 * sigma * sigma)) for m in range(-images, images + 1))
    return np.outer(gx, gy)


def periodic_1d_cosine(seed: int = 1, M: int = 128, dt: float = 1e-2, nsteps: int = 100,
                       amp: float = 5.0) -> Instance:
    """1D periodic workload: u0 = normalised exp(-x^2/(2*0.3^2)) e^{3ix};
    V(x,t) = (1 + 0.5 sin 2t) sum_{m=1..4} a_m cos(m x), a_m ~ U[-amp, amp]."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-amp, amp, size=4)
    x = periodic_grid(M)
    u0 = np.exp(-x ** 2 / (2.0 * 0.3 ** 2)) * np.exp(3j * x)
    u0 = u0 / _grid_norm(u0, 2.0 * math.pi / M)
    V0 = sum(a[m - 1] * np.cos(m * x) for m in range(1, 5))
    return Instance(PERIODIC, (M,), u0.astype(np.complex128), V0.astype(np.float64),
                    lambda t: 1.0 + 0.5 * np.sin(2.0 * np.asarray(t, dtype=np.float64)),
                    None, dt, nsteps, name=f"periodic_1d_cosine_M{M}")


def periodic_2d_wells(seed: int = 2, M: int = 512, dt: float = 1e-3, nsteps: int = 2000,
                      T_pulse: Optional[float] = None, A0: float = 2.0, omega: float = 10.0) -> Instance:
    """2D periodic workload on [-pi,pi]^2: u0 = normalised sum of 3 Gaussians
    (sigma ~ U[0.2,0.4], centres ~ U[-1.5,1.5]^2, phases ~ U[0,2pi)); V0 = sum
    of 4 attractive wells -depth exp(-|x-c|^2/(2 sigma^2)), depth ~ U[5,20],
    sigma ~ U[0.3,0.6], centres ~ U[-1.5,1.5]^2; both summed over lattice
    images |m|<=3 so that they are smooth and periodic.  A(t) = A0
    sin^2(pi t/T_pulse) sin(omega t) (1,0) with T_pulse = nsteps*dt by default."""
    rng = np.random.default_rng(seed)
    x = periodic_grid(M)
    X, Y = np.meshgrid(x, x, indexing="ij")
    u0 = np.zeros((M, M), dtype=np.complex128)
    for _ in range(3):
        s = rng.uniform(0.2, 0.4)
        cx, cy = rng.uniform(-1.5, 1.5, size=2)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        u0 += np.exp(1j * ph) * _periodised_gaussian_2d(X, Y, cx, cy, s)
    u0 = u0 / _grid_norm(u0, 2.0 * math.pi / M)
    V0 = np.zeros((M, M), dtype=np.float64)
    for _ in range(4):
        depth = rng.uniform(5.0, 20.0)
        s = rng.uniform(0.3, 0.6)
        cx, cy = rng.uniform(-1.5, 1.5, size=2)
        V0 -= depth * _periodised_gaussian_2d(X, Y, cx, cy, s)
    Tp = nsteps * dt if T_pulse is None else T_pulse
    pulse = Pulse(A0, omega, Tp, (1.0, 0.0))
    return Instance(PERIODIC, (M, M), u0, V0, _const_one, pulse, dt, nsteps,
                    name=f"periodic_2d_wells_M{M}")


def _periodised_gaussian_1d(x, c, sigma, images=3):
    L = 2.0 * math.pi
    return sum(np.exp(-(x - c - L * m) ** 2 / (2.0 * sigma * sigma)) for m in range(-images, images + 1))


def periodic_3d_wells(seed: int = 2, M: int = 128, dt: float = 1e-3, nsteps: int = 500,
                      A0: float = 2.0, omega: float = 10.0) -> Instance:
    """3D periodic workload on [-pi,pi]^3 shaped like the 2D wells workload:
    u0 = normalised sum of 3 Gaussians (sigma ~ U[0.3,0.5], centres ~
    U[-1,1]^3, random phases); V0 = sum of 4 attractive wells -depth
    exp(-|x-c|^2/(2 sigma^2)), depth ~ U[5,20], sigma ~ U[0.4,0.7], centres ~
    U[-1,1]^3; each Gaussian is a product of 1D lattice-image sums (|m| <= 3),
    so both are smooth and periodic.  A(t) = A0 sin^2(pi t/T) sin(omega t)
    (1,0,0), T = nsteps dt."""
    rng = np.random.default_rng([seed, 3])
    x = periodic_grid(M)

    def gauss(c, s):
        g = [_periodised_gaussian_1d(x, c[a], s) for a in range(3)]
        return g[0][:, None, None] * g[1][None, :, None] * g[2][None, None, :]

    u0 = np.zeros((M, M, M), dtype=np.complex128)
    for _ in range(3):
        s = rng.uniform(0.3, 0.5)
        c = rng.uniform(-1.0, 1.0, size=3)
        u0 += np.exp(1j * rng.uniform(0.0, 2.0 * math.pi)) * gauss(c, s)
    h = 2.0 * math.pi / M
    u0 = u0 / math.sqrt(float(np.sum(np.abs(u0) ** 2)) * h ** 3)
    V0 = np.zeros((M, M, M), dtype=np.float64)
    for _ in range(4):
        depth = rng.uniform(5.0, 20.0)
        s = rng.uniform(0.4, 0.7)
        c = rng.uniform(-1.0, 1.0, size=3)
        V0 -= depth * gauss(c, s)
    pulse = Pulse(A0, omega, nsteps * dt, (1.0, 0.0, 0.0))
    return Instance(PERIODIC, (M, M, M), u0, V0, _const_one, pulse, dt, nsteps, name=f"periodic_3d_wells_M{M}")


BATCH_SIZES = tuple(2 ** p for p in range(8, 15))   # 256 .. 16384


def periodic_1d_batch_member(i: int, seed: int = 4, dt: float = 1e-3, nsteps: int = 1000,
                             sizes: Sequence[int] = BATCH_SIZES) -> Instance:
    """Member i of the uneven 1D batch: N drawn uniformly from `sizes`; V = 4
    cosine modes with a_m ~ U[-10,10]; pulse amplitude A0 ~ U[0,3], omega=10;
    u0 = Gaussian with sigma ~ U[0.2,0.4], centre ~ U[-1,1], k0 ~ U[-5,5]."""
    rng = np.random.default_rng([seed, i])
    M = int(sizes[int(rng.integers(0, len(sizes)))])
    a = rng.uniform(-10.0, 10.0, size=4)
    A0 = rng.uniform(0.0, 3.0)
    s = rng.uniform(0.2, 0.4)
    c = rng.uniform(-1.0, 1.0)
    k0 = rng.uniform(-5.0, 5.0)
    x = periodic_grid(M)
    L = 2.0 * math.pi
    g = sum(np.exp(-(x - c - L * m) ** 2 / (2.0 * s * s)) for m in range(-3, 4))
    u0 = g * np.exp(1j * k0 * x)
    u0 = u0 / _grid_norm(u0, L / M)
    V0 = sum(a[m - 1] * np.cos(m * x) for m in range(1, 5))
    pulse = Pulse(A0, 10.0, nsteps * dt, (1.0,))
    return Instance(PERIODIC, (M,), u0.astype(np.complex128), V0.astype(np.float64), _const_one,
                    pulse, dt, nsteps, name=f"periodic_1d_batch_{i}_M{M}")


def random_periodic(shape, seed: int, dt: float, nsteps: int, vamp: float = 5.0,
                    pulse: Optional[Pulse] = None, vfac: Optional[Callable] = None,
                    nmodes: int = 3) -> Instance:
    """Small smooth random periodic problem for parity tests: u0 and V0 are
    random trigonometric polynomials of degree `nmodes` per dimension."""
    rng = np.random.default_rng(seed)
    d = len(shape)
    grids = np.meshgrid(*[periodic_grid(M) for M in shape], indexing="ij")
    u0 = np.zeros(shape, dtype=np.complex128)
    V0 = np.zeros(shape, dtype=np.float64)
    for idx in np.ndindex(*([2 * nmodes + 1] * d)):
        k = [i - nmodes for i in idx]
        ph = sum(kk * g for kk, g in zip(k, grids))
        w = math.exp(-0.5 * sum(kk * kk for kk in k))
        u0 += w * (rng.normal() + 1j * rng.normal()) * np.exp(1j * ph)
        V0 += vamp * w * (rng.normal() * np.cos(ph) + rng.normal() * np.sin(ph))
    h = 2.0 * math.pi / shape[0]
    u0 = u0 / _grid_norm(u0, h)
    return Instance(PERIODIC, tuple(shape), u0, V0, vfac or _const_one, pulse, dt, nsteps,
                    name=f"random_periodic_{'x'.join(map(str, shape))}")


def bump_window(X: Sequence[np.ndarray], radius: float = 0.95) -> np.ndarray:
    """exp(1 - 1/(1 - r^2)) for r = |x| / radius < 1, else 0 (C-infinity, compact)."""
    r2 = sum(x * x for x in X) / (radius * radius)
    out = np.zeros_like(r2)
    inside = r2 < 1.0
    out[inside] = np.exp(1.0 - 1.0 / (1.0 - r2[inside]))
    return out


def free_bump_gaussians(shape=(256, 256), seed: int = 3, dt: float = 5e-4, nsteps: int = 2000,
                        T_pulse: Optional[float] = None, A0: float = 2.0, omega: float = 10.0,
                        direction: Optional[Sequence[float]] = None, n_u: int = 3, n_v: int = 4,
                        vfac: Optional[Callable] = None) -> Instance:
    """Free-space workload on [-1,1]^d: u0 = normalised sum of n_u Gaussians
    (sigma ~ U[0.08,0.15], centres ~ U[-0.4,0.4]^d, phases ~ U[0,2pi)) times
    the bump window; V0 = -sum of n_v wells depth exp(-|x-c|^2/(2 sigma^2))
    (depth ~ U[5,20], sigma ~ U[0.08,0.15], centres ~ U[-0.4,0.4]^d) times the
    window.  A(t) = A0 sin^2(pi t / T_pulse) sin(omega t) along `direction`
    (default (1, 0, ..)), T_pulse = nsteps dt by default."""
    rng = np.random.default_rng(seed)
    d = len(shape)
    X = np.meshgrid(*[free_grid(M) for M in shape], indexing="ij")
    win = bump_window(X)

    def gauss(c, s):
        return np.exp(-sum((x - cc) ** 2 for x, cc in zip(X, c)) / (2.0 * s * s))

    u0 = np.zeros(tuple(shape), dtype=np.complex128)
    for _ in range(n_u):
        s = rng.uniform(0.08, 0.15)
        c = rng.uniform(-0.4, 0.4, size=d)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        u0 += np.exp(1j * ph) * gauss(c, s)
    u0 *= win
    u0 = u0 / _grid_norm(u0, 2.0 / shape[0])
    V0 = np.zeros(tuple(shape), dtype=np.float64)
    for _ in range(n_v):
        depth = rng.uniform(5.0, 20.0)
        s = rng.uniform(0.08, 0.15)
        c = rng.uniform(-0.4, 0.4, size=d)
        V0 -= depth * gauss(c, s)
    V0 *= win
    Tp = nsteps * dt if T_pulse is None else T_pulse
    dirn = tuple(direction) if direction is not None else (1.0,) + (0.0,) * (d - 1)
    pulse = Pulse(A0, omega, Tp, dirn) if A0 else None
    return Instance(FREE, tuple(shape), u0, V0, vfac or _const_one, pulse, dt, nsteps,
                    name=f"free_bump_gaussians_{'x'.join(map(str, shape))}")


def _moving_gaussians(X: Sequence[np.ndarray], wells, t: float, period: Optional[float], images: int) -> np.ndarray:
    """-sum_w depth_w exp(-|x - c_w - v_w t|^2 / (2 sigma_w^2)), summed over the
    lattice images |m| <= images when `period` is set."""
    out = np.zeros_like(X[0])
    shifts = range(-images, images + 1) if period else (0,)
    for depth, c, v, sigma in wells:
        ctr = [ci + vi * t for ci, vi in zip(c, v)]
        for m in np.ndindex(*([len(shifts)] * len(X))):
            r2 = sum((x - cc - (period or 0.0) * shifts[mi]) ** 2 for x, cc, mi in zip(X, ctr, m))
            out -= depth * np.exp(-r2 / (2.0 * sigma * sigma))
    return out


def well_ground_state_coeffs(V0: float, beta: float, K: int = 96):
    """Ground state of -w'' + V w = E w on [-pi, pi] with V the periodic
    extension of -V0 exp(-x^2 / (2 beta^2)): Fourier-Galerkin on |k| <= K with
    the exact coefficients of the periodised Gaussian,
    V^_m = -V0 beta / sqrt(2 pi) exp(-beta^2 m^2 / 2); dense symmetric
    eigensolve.  Returns (E, k, c) with w(x) = sum_k c_k e^{i k x}, normalised
    to unit L2 norm on [-pi, pi]."""
    k = np.arange(-K, K + 1)
    m = k[:, None] - k[None, :]
    H = -V0 * beta / math.sqrt(2.0 * math.pi) * np.exp(-0.5 * beta * beta * m * m)
    H = H + np.diag(k.astype(np.float64) ** 2)
    E, vec = np.linalg.eigh(H)
    c = vec[:, 0] / math.sqrt(2.0 * math.pi)
    return float(E[0]), k, c.astype(np.complex128)


def moving_well_1d(c: float = 30.0, M: int = 256, nsteps: int = 3200, T: float = 2.0 * math.pi / 15.0,
                   V0: float = 300.0, beta: float = 0.2, x0: float = 0.0, u_shift: float = 0.0,
                   K: int = 96) -> Instance:
    """Moving periodic Gaussian well (Example 1): V(x, t) = -V0 sum_m
    exp(-(x - 2 pi m - x0 - c t)^2 / (2 beta^2)), A = 0, u0 = the normalised
    ground state of V(., 0) times e^{i u_shift x} (u_shift = c / 2 gives the
    Galilean-boosted state that the well carries exactly when c / 2 is an
    integer).  Defaults: V0 = 300, beta = 0.2, T = 2 pi / 15."""
    x = periodic_grid(M)
    E, k, coef = well_ground_state_coeffs(V0, beta, K)
    u0 = (np.exp(1j * np.outer(x - x0, k)) @ coef) * np.exp(1j * u_shift * x)
    wells = [(V0, (x0,), (c,), beta)]

    def Vt(t, _x=(x,), _w=wells):
        return _moving_gaussians(_x, _w, float(t), 2.0 * math.pi, 3)

    dt = T / nsteps
    return Instance(PERIODIC, (M,), u0.astype(np.complex128), Vt(0.0), _const_one, None, dt, nsteps,
                    name=f"moving_well_1d_c{c:g}_M{M}", Vt=Vt)


def free_moving_well(M: int = 256, V0: float = 3000.0, beta: float = 0.06, x0: float = -0.1, c: float = 1.0,
                     T: float = 0.02, nsteps: int = 800, K: int = 320) -> Instance:
    """Free space on [-1,1]: a deep Gaussian well V(x, t) = -V0 exp(-(x - x0 -
    c t)^2 / (2 beta^2)) moving at speed c, A = 0; u0 = its ground state (the
    Fourier-Galerkin eigensolve of `well_ground_state_coeffs`, whose [-pi, pi]
    box holds the state's exponentially small tails) boosted by e^{i c x / 2},
    the state the well carries along (below 1e-15 at x = +-1 for the defaults)."""
    x = free_grid(M)
    E, k, coef = well_ground_state_coeffs(V0, beta, K)
    u0 = (np.exp(1j * np.outer(x - x0, k)) @ coef) * np.exp(0.5j * c * x)

    def Vt(t, _x=x):
        return -V0 * np.exp(-(_x - x0 - c * float(t)) ** 2 / (2.0 * beta * beta))

    return Instance(FREE, (M,), u0.astype(np.complex128), Vt(0.0), _const_one, None, T / nsteps, nsteps,
                    name=f"free_moving_well_M{M}", Vt=Vt)


def moving_separable_wells_2d(M: int = 64, nsteps: int = 200, T: float = 0.2, wells=((40.0, 0.45), (60.0, 0.5)),
                              c=(4.0, -2.0), K: int = 96) -> Instance:
    """2D periodic V(x, y, t) = W_1(x - c_x t) + W_2(y - c_y t), W_a the
    periodised Gaussian well -V0_a exp(-s^2 / (2 beta_a^2)); A = 0; u0 = the
    product of the two wells' ground states boosted by e^{i c.x / 2} (the state
    the wells carry along when c_x / 2, c_y / 2 are integers)."""
    x = periodic_grid(M)
    X, Y = np.meshgrid(x, x, indexing="ij")
    g = [well_ground_state_coeffs(V0, b, K) for V0, b in wells]
    w = [np.exp(1j * np.outer(x, k)) @ coef for _, k, coef in g]
    u0 = np.outer(w[0], w[1]) * np.exp(0.5j * (c[0] * X + c[1] * Y))
    mw = [[(V0, (0.0,), (cc,), b)] for (V0, b), cc in zip(wells, c)]

    def Vt(t, _x=(x,), _m=mw):
        a = _moving_gaussians(_x, _m[0], float(t), 2.0 * math.pi, 3)
        b = _moving_gaussians(_x, _m[1], float(t), 2.0 * math.pi, 3)
        return a[:, None] + b[None, :]

    return Instance(PERIODIC, (M, M), u0.astype(np.complex128), Vt(0.0), _const_one, None, T / nsteps, nsteps,
                    name=f"moving_separable_wells_2d_M{M}", Vt=Vt)


def example1_sweep(count: int, c: float, seed: int = 11, M: int = 512, nsteps: int = 3200,
                   T: float = 2.0 * math.pi / 15.0, V0: float = 300.0, beta: float = 0.2):
    """A sweep over initial states for one well speed of Example 1: the well
    instance (its V(x, t) is shared) and `count` initial states, the ground
    state displaced by s grid points (s ~ U{-12..12}) and kicked by e^{i k0 x}
    (k0 ~ U{-6..6}).  Returns (instance, u0 array [count, M])."""
    base = moving_well_1d(c=c, M=M, nsteps=nsteps, T=T, V0=V0, beta=beta)
    rng = np.random.default_rng([seed, int(round(c * 1000))])
    x = periodic_grid(M)
    shifts = rng.integers(-12, 13, size=count)
    kicks = rng.integers(-6, 7, size=count)
    u0 = np.stack([np.roll(base.u0, int(s)) * np.exp(1j * int(k) * x) for s, k in zip(shifts, kicks)])
    return base, u0.astype(np.complex128)


def moving_wells_2d(seed: int = 6, M: int = 64, dt: float = 1e-3, nsteps: int = 40, speed: float = 8.0,
                    A0: float = 2.0, omega: float = 10.0) -> Instance:
    """2D periodic wells drifting at constant velocity (a non-separable V):
    the 2D wells workload's u0 and pulse, its four wells with velocities
    ~ speed * U[-1,1]^2."""
    base = periodic_2d_wells(seed=seed, M=M, dt=dt, nsteps=nsteps, A0=A0, omega=omega)
    rng = np.random.default_rng([seed, 77])
    x = periodic_grid(M)
    X = tuple(np.meshgrid(x, x, indexing="ij"))
    wells = [(rng.uniform(5.0, 20.0), tuple(rng.uniform(-1.5, 1.5, size=2)), tuple(speed * rng.uniform(-1, 1, size=2)),
              rng.uniform(0.3, 0.6)) for _ in range(4)]

    def Vt(t, _X=X, _w=wells):
        return _moving_gaussians(_X, _w, float(t), 2.0 * math.pi, 3)

    return Instance(PERIODIC, (M, M), base.u0, Vt(0.0), _const_one, base.pulse, dt, nsteps,
                    name=f"moving_wells_2d_M{M}", Vt=Vt)


def free_moving_wells(shape=(64,), seed: int = 7, dt: float = 1e-3, nsteps: int = 40, speed: float = 2.0,
                      A0: float = 20.0, omega: float = 30.0) -> Instance:
    """Free space on [-1,1]^d: the bump-windowed u0 and pulse of the
    free-space workload with four wells drifting at velocities
    ~ speed * U[-1,1]^d, the wells times the bump window at every t."""
    base = free_bump_gaussians(shape, seed=seed, dt=dt, nsteps=nsteps, A0=A0, omega=omega)
    d = len(shape)
    rng = np.random.default_rng([seed, 78])
    X = tuple(np.meshgrid(*[free_grid(M) for M in shape], indexing="ij"))
    win = bump_window(X)
    wells = [(rng.uniform(5.0, 20.0), tuple(rng.uniform(-0.4, 0.4, size=d)), tuple(speed * rng.uniform(-1, 1, size=d)),
              rng.uniform(0.08, 0.15)) for _ in range(4)]

    def Vt(t, _X=X, _w=wells, _win=win):
        return _moving_gaussians(_X, _w, float(t), None, 0) * _win

    return Instance(FREE, tuple(shape), base.u0, Vt(0.0), _const_one, base.pulse, dt, nsteps,
                    name=f"free_moving_wells_{'x'.join(map(str, shape))}", Vt=Vt)


def serve_requests(seed: int = 5, rate: float = 200.0, duration: float = 10.0, T_range=(0.5, 2.0),
                   dt_range=(2e-4, 2e-3), sizes_1d=tuple(2 ** p for p in range(10, 15)),
                   sizes_2d=tuple(2 ** p for p in range(7, 11)), sizes_free=tuple(2 ** p for p in range(6, 9))):
    """Seeded request stream: Poisson arrivals (mean `rate` per second over
    `duration` s); each request is 1D periodic, 2D periodic or 2D free space
    with probability 1/3 each, its size drawn uniformly from the class's
    sizes, T ~ U[T_range], dt log-uniform on dt_range, nsteps = round(T/dt),
    data as in the 1D batch, 2D wells and free-space workloads.  Returns
    [(arrival, class, Instance)]."""
    rng = np.random.default_rng(seed)
    t, out, i = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        cls = int(rng.integers(0, 3))
        T = rng.uniform(*T_range)
        dt = float(math.exp(rng.uniform(math.log(dt_range[0]), math.log(dt_range[1]))))
        n = max(8, int(round(T / dt)))
        sub = 100000 * seed + i
        if cls == 0:
            M = int(sizes_1d[int(rng.integers(0, len(sizes_1d)))])
            inst = periodic_1d_batch_member(sub, seed=seed, dt=dt, nsteps=n, sizes=(M,))
            kind = "1d"
        elif cls == 1:
            M = int(sizes_2d[int(rng.integers(0, len(sizes_2d)))])
            inst = periodic_2d_wells(seed=sub, M=M, dt=dt, nsteps=n)
            kind = "2d"
        else:
            M = int(sizes_free[int(rng.integers(0, len(sizes_free)))])
            inst = free_bump_gaussians((M, M), seed=sub, dt=dt, nsteps=n)
            kind = "free"
        out.append((t, kind, inst))
        i += 1
