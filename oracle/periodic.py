"""Periodic marching scheme, plain FP64 (oracle; test infrastructure only).

Follows Sec. 2 of Kaye-Barnett-Greengard in the paper's own order:

* grid x_j = -pi + 2 pi j/M, modes k = -M/2 .. M/2-1 per dimension (Sec. 2.1);
* forward DFT  f^_k = (1/M) sum_j e^{-2 pi i j k/M} f_j       (eq. ftperdisc),
  inverse      f_j  = sum_k e^{+2 pi i j k/M} f^_k           (eq. utrapkdisc),
  both as direct O(M^2) sums per dimension (a dense matrix product);
* trapezoidal step (eq. utrapkdisc):
  u(t) = IDFT[ P(t,dt) (u^(t-dt) - i dt/2 (Vu)^(t-dt)) ] / (1 + i dt/2 V(t));
* n-th order implicit Adams step (eq. uadamsk):
  u(t) = IDFT[ P(t,dt) u^(t-dt) - i dt sum_{j=1}^{n-1} mu_j P(t, j dt) (Vu)^(t-j dt) ]
         / (1 + i mu_0 dt V(t));
  with P(t, s) = exp(-i |k|^2 s + i k.(phi(t) - phi(t-s))) evaluated directly;
* start-up (Sec. 2.2): iterated Richardson extrapolation of trapezoidal
  chains with 1, 2, 4, ... sub-steps, skipping odd orders; by default n-1
  start-up steps (the paper's "seven" for n = 8; reading C1).

The state kept between steps is the physical solution u(x_j, t_n) and the
history of (Vu)^ at previous steps, exactly as the formulas are written.
"""
from __future__ import annotations

import math
from typing import Callable, Optional

import numpy as np

from . import adams


def wavenumbers(M: int) -> np.ndarray:
    """k = -M/2 .. M/2-1 (Sec. 2.1; the paper's truncation, Nyquist at -M/2)."""
    if M % 2:
        raise ValueError("M must be even")
    return np.arange(-M // 2, M // 2, dtype=np.float64)


def dft_matrices(M: int):
    """Dense forward (1/M) e^{-2 pi i j k/M} and inverse e^{+2 pi i j k/M} matrices.

    Rows of F / columns of G are ordered k = -M/2 .. M/2-1.  The integer
    product j k is reduced mod M before scaling so that the angles are exact.
    """
    j = np.arange(M, dtype=np.int64)
    k = np.arange(-M // 2, M // 2, dtype=np.int64)
    jk = np.mod(np.outer(k, j), M).astype(np.float64)          # [k, j]
    ang = 2.0 * math.pi * jk / M
    F = (np.cos(ang) - 1j * np.sin(ang)) / M                   # [k, j]
    G = (np.cos(ang) + 1j * np.sin(ang)).T.copy()              # [j, k]
    return F, G


def rel_l2(u: np.ndarray, ref: np.ndarray) -> float:
    """Relative L2 error with the left-endpoint grid rule (eq. l2err); the
    cell volume cancels in the ratio."""
    return float(np.sqrt(np.sum(np.abs(u - ref) ** 2) / np.sum(np.abs(ref) ** 2)))


class PeriodicOracle:
    """Direct implementation of the periodic scheme for d = 1 or 2.

    Parameters
    ----------
    shape : grid points per dimension (each even).
    dt    : time step.
    V0, vfac : V(x, t) = vfac(t) * V0(x) (real); or V0 a callable t -> V(., t)
               on the grid (any real potential, the problem of Sec. 1 with
               general V(x, t)), vfac then unused.
    phi   : callable t -> array(d), phi(t) = int_0^t A.
    order : Adams order n (even, >= 2).
    n_startup : number of Richardson start-up steps (default n - 1).
    transform : "direct" (the dense O(M^2) sums of eqs. ftperdisc / utrapkdisc)
                or "fft" (the same DFT pair through numpy's FFT, a library
                primitive, for grids where the dense matrices do not fit in
                memory; pinned against "direct").
    """

    def __init__(self, shape, dt: float, V0: np.ndarray, vfac: Callable, phi: Callable,
                 order: int = 8, n_startup: Optional[int] = None, transform: str = "direct"):
        self.shape = tuple(int(m) for m in shape)
        self.d = len(self.shape)
        if order < 2 or order % 2:
            raise ValueError("order must be even and >= 2")
        self.dt = float(dt)
        self.Vt = V0 if callable(V0) else None
        self.V0 = None if callable(V0) else np.asarray(V0, dtype=np.float64)
        self.vfac = vfac
        self.phi = phi
        self.order = order
        self.n_startup = order - 1 if n_startup is None else int(n_startup)
        if self.n_startup < order - 2:
            raise ValueError("need at least order-2 start-up steps")
        self.mu = adams.weights(order)
        if transform not in ("direct", "fft"):
            raise ValueError("transform: direct or fft")
        self.transform = transform
        if transform == "direct":
            mats = [dft_matrices(M) for M in self.shape]
            self.F = [m[0] for m in mats]
            self.G = [m[1] for m in mats]
        ks = [wavenumbers(M) for M in self.shape]
        self.k = np.meshgrid(*ks, indexing="ij")                 # list of d arrays
        self.ksq = sum(kk * kk for kk in self.k)

    # -- transforms (direct sums, one dimension at a time) ---------------------
    def _apply(self, mats, f):
        out = np.asarray(f, dtype=np.complex128)
        for ax, Mx in enumerate(mats):
            out = np.moveaxis(np.tensordot(Mx, out, axes=([1], [ax])), 0, ax)
        return out

    def fwd(self, f):
        """(1/M^d) sum_j e^{-2 pi i j.k/M} f_j  (eq. ftperdisc, per dimension)."""
        if self.transform == "fft":          # modes ordered k = -M/2 .. M/2-1, as the dense rows
            axes = tuple(range(self.d))
            return np.fft.fftshift(np.fft.fftn(np.asarray(f, dtype=np.complex128), axes=axes), axes=axes) / float(
                np.prod(self.shape))
        return self._apply(self.F, f)

    def inv(self, fh):
        """sum_k e^{+2 pi i j.k/M} f^_k  (eq. utrapkdisc, per dimension)."""
        if self.transform == "fft":
            axes = tuple(range(self.d))
            return np.fft.ifftn(np.fft.ifftshift(np.asarray(fh, dtype=np.complex128), axes=axes), axes=axes) * float(
                np.prod(self.shape))
        return self._apply(self.G, fh)

    # -- problem data ---------------------------------------------------------
    def V(self, t: float) -> np.ndarray:
        if self.Vt is not None:
            return np.asarray(self.Vt(t), dtype=np.float64)
        return float(self.vfac(t)) * self.V0

    def P(self, t: float, s: float) -> np.ndarray:
        """Spectral Green's function over [t-s, t]:
        exp(-i |k|^2 s + i k.(phi(t) - phi(t-s)))  (eq. uhatkrecur)."""
        dphi = np.asarray(self.phi(t), dtype=np.float64) - np.asarray(self.phi(t - s), dtype=np.float64)
        arg = -self.ksq * s + sum(self.k[a] * dphi[a] for a in range(self.d))
        return np.cos(arg) + 1j * np.sin(arg)

    # -- steps ----------------------------------------------------------------
    def trapezoid_step(self, v: np.ndarray, t0: float, h: float) -> np.ndarray:
        """One step of eq. utrapkdisc from time t0 to t0 + h."""
        t1 = t0 + h
        g = self.P(t1, h) * (self.fwd(v) - 0.5j * h * self.fwd(self.V(t0) * v))
        return self.inv(g) / (1.0 + 0.5j * h * self.V(t1))

    def richardson_step(self, u_prev: np.ndarray, t0: float) -> np.ndarray:
        """Iterated Richardson extrapolation of trapezoidal chains (Sec. 2.2).

        Chains c = 0..L-1 take 2^c sub-steps of dt/2^c (L = order/2); level l
        combines neighbours with factor 4^l (only even error powers)."""
        L = self.order // 2
        table = []
        for c in range(L):
            m = 2 ** c
            h = self.dt / m
            v = u_prev
            for s in range(m):
                v = self.trapezoid_step(v, t0 + s * h, h)
            table.append(v)
        for lev in range(1, L):
            f = 4.0 ** lev
            table = [(f * table[c + 1] - table[c]) / (f - 1.0) for c in range(len(table) - 1)]
        return table[0]

    def adams_step(self, u_prev: np.ndarray, t: float, vu_hist: dict, n: int) -> np.ndarray:
        """One step of eq. uadamsk producing u(t_n), t = n dt."""
        dt = self.dt
        g = self.P(t, dt) * self.fwd(u_prev)
        for j in range(1, self.order):
            g = g - 1j * dt * self.mu[j] * self.P(t, j * dt) * vu_hist[n - j]
        return self.inv(g) / (1.0 + 1j * self.mu[0] * dt * self.V(t))

    # -- driver ---------------------------------------------------------------
    def solve(self, u0: np.ndarray, nsteps: int, keep=None):
        """March u0 over `nsteps` steps of size dt.

        Returns u(t_nsteps); if `keep` is a collection of step indices, also
        returns {n: u(t_n)} for those indices."""
        u = np.asarray(u0, dtype=np.complex128)
        hist = {0: self.fwd(self.V(0.0) * u)}
        kept = {}
        if keep is not None and 0 in keep:
            kept[0] = u.copy()
        for n in range(1, nsteps + 1):
            t = n * self.dt
            if n <= self.n_startup:
                u = self.richardson_step(u, (n - 1) * self.dt)
            else:
                u = self.adams_step(u, t, hist, n)
            hist[n] = self.fwd(self.V(t) * u)
            hist.pop(n - self.order, None)
            if keep is not None and n in keep:
                kept[n] = u.copy()
        return (u, kept) if keep is not None else u


def oracle_for(inst, order: int = 8, n_startup: Optional[int] = None, transform: str = "direct") -> PeriodicOracle:
    """Build the oracle for a synth.Instance (phi in closed form for its pulse)."""
    from .fields import phi_callable
    return PeriodicOracle(inst.shape, inst.dt, inst.V0, inst.vfac,
                          phi_callable(inst.pulse, inst.dim), order=order, n_startup=n_startup, transform=transform)
