"""Free-space (complex-frequency) marching scheme, plain FP64 (oracle; test
infrastructure only).

Sec. 3.4 and Remark highorderfs, in the paper's order:
  * grid x_j = -1 + 2 (j-1)/M, j = 1..M per dimension (Sec. 3.4);
  * nodes zeta_k and weights w_k on Gamma_K from `gamma.GammaRule`;
  * forward transform  f^(zeta_k) = (2/M)^d sum_j e^{-i zeta_k . x_j} f_j     (eq. fzdft)
    inverse          f(x_j)     = (1/2pi)^d sum_k w_k e^{i zeta_k . x_j} f^_k (eq. uciftdisc)
    as direct sums per dimension (dense matrices; d = 2 is the tensor product);
  * P(t, s) = exp(-i zeta.zeta s + i zeta.(phi(t) - phi(t-s)))  (eq. uhatxirecur
    with xi -> zeta, |xi|^2 -> zeta.zeta);
  * trapezoidal step (eqs. uhatzfd, utrapzfd): u(t) from u^(t-h), (Vu)^(t-h);
    (Vu)^(t) = DFT(V u(t)); u^(t) = P (u^ - i h/2 (Vu)^(t-h)) - i h/2 (Vu)^(t);
  * n-th order implicit Adams (Remark highorderfs), same formulas as Sec. 2.2;
  * start-up by iterated Richardson extrapolation applied to both u and u^
    (Remark highorderfs); then (Vu)^(t_n) = DFT(V(t_n) u_combined).
The state is (u^ on Gamma, u on the grid, history of (Vu)^); u is never
obtained by transforming u^ (it would need u outside [-1,1]^d).
"""
from __future__ import annotations

import math
from typing import Callable, Optional, Sequence

import numpy as np

from . import adams
from .gamma import GammaRule


def free_grid(M: int) -> np.ndarray:
    return -1.0 + 2.0 * np.arange(M, dtype=np.float64) / M


def ctype_chebyshev(rule: GammaRule, NT: int):
    """C-type transforms through Chebyshev interpolants (Sec. 4.1, eqs.
    expintrpm and expintrpp), for one dimension of `rule`.

    On Gamma_2, zeta = (1 - i) tau with tau in [-H, H], so
        e^{-i zeta x_j} = e^{-tau x_j} e^{-i tau x_j} ~ sum_l lambda_{l,j} T_l^H(tau),
        e^{+i zeta x_j} = e^{+tau x_j} e^{+i tau x_j} ~ sum_l rho_{j,l} T_l^H(tau),
    with T_l^H(tau) = T_l(tau / H) and each interpolant the polynomial of degree
    NT - 1 through the values at the Chebyshev points tau_m = H cos(pi (m + 1/2) / NT).
    Changing the order of summation gives
        f^_k = (2/M) sum_l T_l^H(tau_k) sum_j lambda_{l,j} f_j         (forward, C nodes)
        f_j  = (1/2pi) sum_l rho_{j,l} sum_k T_l^H(tau_k) w_k f^_k    (inverse, C nodes)
    Returns (fwd, inv): fwd(f) -> the NC C-node values, inv(fhat_C) -> M grid
    values, with the same scalings as eqs. fzdft / uciftdisc."""
    M, H = rule.M, rule.H
    x = free_grid(M)
    theta = math.pi * (np.arange(NT) + 0.5) / NT
    tau_m = H * np.cos(theta)
    Cmat = np.cos(np.outer(np.arange(NT), theta))                       # [l, m] = T_l(cos theta_m)
    g_minus = np.exp(-(1.0 + 1.0j) * np.outer(tau_m, x))                # [m, j]
    g_plus = np.exp((1.0 + 1.0j) * np.outer(tau_m, x))
    lam = (2.0 / NT) * (Cmat @ g_minus)                                 # [l, j]
    rho = (2.0 / NT) * (Cmat @ g_plus)
    lam[0] *= 0.5
    rho[0] *= 0.5
    tau_k = rule.tau_c
    Tk = np.cos(np.outer(np.arccos(np.clip(tau_k / H, -1.0, 1.0)), np.arange(NT)))   # [k, l] = T_l^H(tau_k)
    w_c = rule.blocks["C"][1]

    def fwd(f):
        return (2.0 / M) * (Tk @ (lam @ np.asarray(f, dtype=np.complex128)))

    def inv(fh_c):
        return (rho.T @ (Tk.T @ (w_c * np.asarray(fh_c, dtype=np.complex128)))) / (2.0 * math.pi)

    return fwd, inv


class FreeSpaceOracle:
    """Direct implementation of the free-space scheme for d = 1 or 2.

    rules: one GammaRule per dimension.  V(x,t) = vfac(t) V0(x), or V0 a
    callable t -> V(., t) on the grid (general V, vfac unused); phi(t) -> (d,).
    """

    def __init__(self, rules: Sequence[GammaRule], dt: float, V0: np.ndarray, vfac: Callable, phi: Callable,
                 order: int = 8, n_startup: Optional[int] = None):
        self.rules = list(rules)
        self.d = len(self.rules)
        self.dt = float(dt)
        self.Vt = V0 if callable(V0) else None
        self.V0 = None if callable(V0) else np.asarray(V0, dtype=np.float64)
        self.vfac = vfac
        self.phi = phi
        self.order = order
        self.n_startup = order - 1 if n_startup is None else int(n_startup)
        self.mu = adams.weights(order)
        self.F, self.G = [], []
        for r in self.rules:
            x = free_grid(r.M)
            E = np.exp(-1j * np.outer(r.zeta, x))                       # [k, j]
            self.F.append((2.0 / r.M) * E)
            self.G.append(np.exp(1j * np.outer(x, r.zeta)) * (r.w[None, :] / (2.0 * math.pi)))  # [j, k]
        Z = np.meshgrid(*[r.zeta for r in self.rules], indexing="ij")
        self.Z = Z
        self.zz = sum(z * z for z in Z)

    def _apply(self, mats, f):
        out = np.asarray(f, dtype=np.complex128)
        for ax, Mx in enumerate(mats):
            out = np.moveaxis(np.tensordot(Mx, out, axes=([1], [ax])), 0, ax)
        return out

    def fwd(self, f):
        """(2/M)^d sum_j e^{-i zeta.x_j} f_j (eq. fzdft)."""
        return self._apply(self.F, f)

    def inv(self, fh):
        """(1/2pi)^d sum_k w_k e^{i zeta_k.x_j} f^_k (eq. uciftdisc)."""
        return self._apply(self.G, fh)

    def V(self, t: float) -> np.ndarray:
        if self.Vt is not None:
            return np.asarray(self.Vt(t), dtype=np.float64)
        return float(self.vfac(t)) * self.V0

    def P(self, t: float, s: float) -> np.ndarray:
        dphi = np.asarray(self.phi(t), dtype=np.float64) - np.asarray(self.phi(t - s), dtype=np.float64)
        arg = -self.zz * s + sum(self.Z[a] * dphi[a] for a in range(self.d))
        return np.exp(1j * arg)

    # -- steps ----------------------------------------------------------------
    def trapezoid_step(self, uh, vuh, t0: float, h: float):
        """eqs. utrapzfd / uhatzfd from t0 to t0 + h; returns (u^, u, (Vu)^)."""
        t1 = t0 + h
        g = self.P(t1, h) * (uh - 0.5j * h * vuh)
        u = self.inv(g) / (1.0 + 0.5j * h * self.V(t1))
        vu1 = self.fwd(self.V(t1) * u)
        return g - 0.5j * h * vu1, u, vu1

    def richardson_step(self, uh, vuh, t0: float):
        L = self.order // 2
        tab_h, tab_u = [], []
        for c in range(L):
            m = 2 ** c
            h = self.dt / m
            a, v = uh, vuh
            for s in range(m):
                a, u, v = self.trapezoid_step(a, v, t0 + s * h, h)
            tab_h.append(a)
            tab_u.append(u)
        for lev in range(1, L):
            f = 4.0 ** lev
            tab_h = [(f * tab_h[c + 1] - tab_h[c]) / (f - 1.0) for c in range(len(tab_h) - 1)]
            tab_u = [(f * tab_u[c + 1] - tab_u[c]) / (f - 1.0) for c in range(len(tab_u) - 1)]
        return tab_h[0], tab_u[0]

    def adams_step(self, uh_prev, t: float, hist: dict, n: int):
        dt = self.dt
        g = self.P(t, dt) * uh_prev
        for j in range(1, self.order):
            g = g - 1j * dt * self.mu[j] * self.P(t, j * dt) * hist[n - j]
        u = self.inv(g) / (1.0 + 1j * self.mu[0] * dt * self.V(t))
        vu = self.fwd(self.V(t) * u)
        return g - 1j * self.mu[0] * dt * vu, u, vu

    def solve(self, u0: np.ndarray, nsteps: int, keep=None):
        """March nsteps steps from u0; returns u(t_n) (and {n: u} for n in keep).
        The final mode state u^ is left in self.last_uhat."""
        u = np.asarray(u0, dtype=np.complex128)
        uh = self.fwd(u)
        hist = {0: self.fwd(self.V(0.0) * u)}
        kept = {}
        if keep is not None and 0 in keep:
            kept[0] = u.copy()
        for n in range(1, nsteps + 1):
            t = n * self.dt
            if n <= self.n_startup:
                uh, u = self.richardson_step(uh, hist[n - 1], (n - 1) * self.dt)
                hist[n] = self.fwd(self.V(t) * u)
            else:
                uh, u, hist[n] = self.adams_step(uh, t, hist, n)
            hist.pop(n - self.order, None)
            if keep is not None and n in keep:
                kept[n] = u.copy()
        self.last_uhat = uh
        return (u, kept) if keep is not None else u
