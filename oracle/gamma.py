"""Quadrature on the deformed contour Gamma (oracle; test infrastructure only).

Sec. 3.3 (eq. gammadef): Gamma = Gamma_1 u Gamma_2 u Gamma_3 with
  Gamma_1: tau + iH (tau < -H),  Gamma_2: tau - i tau (|tau| <= H),  Gamma_3: tau - iH (tau > H),
truncated to |Re zeta| <= K.  Sec. 3.4 ("Quadrature rule on Gamma"):
  * Gamma_3: equispaced nodes H + kappa h + k h, k = 0..NE-1, weight h, plus
    Alpert's p one-sided endpoint corrections H + x_k h with weights h w_k
    (right correction dropped: the integrand has decayed there), with
    h = (K - H) / (NE + 2 kappa - 1)  (reading C3 of the offset);
  * Gamma_1 by the reflection zeta -> -zeta;
  * Gamma_2: dyadically refined composite q-point Gauss-Legendre panels
    a_0 = 0, a_k = H / 2^(n_r - k) (k = 1..n_r) and their mirror images, on the
    parameter tau with d zeta = (1 - i) d tau; n_r = 0 is read as a single
    panel on [-H, H] (reading C2).
Sec. 4.1: K = H + pi M / 2 and nu = 2 (NE + 2 kappa - 1).
Remark Hchoice: H = log(eps / ((1 + ||V||_{2,inf}) eps_m)) / (2 d (1 + phi_max)).

Alpert's node/weight tables are not printed in the paper (only kappa = 7 for
p = 8).  They are derived here from the condition that the corrected rule
    h sum_k w_k f(a + x_k h) + h sum_{j>=0} f(a + (kappa + j) h)
integrates f exactly to order h^(2p): by the Euler-Maclaurin expansion with
Hurwitz-zeta regularisation, sum_k w_k x_k^m = B_{m+1}(kappa)/(m+1) for
m = 0..2p-1 (B the Bernoulli polynomials).  The p-point rule matching 2p
moments is found by Prony's method in exact rational arithmetic (monic
polynomial from the Hankel system), its roots polished by Newton's method in
60-digit decimal arithmetic, and the weights from the Vandermonde system.
"""
from __future__ import annotations

import math
from decimal import Decimal, getcontext
from fractions import Fraction
from functools import lru_cache

import numpy as np

EPS_M = 2.0 ** -52


# ----------------------------------------------------------------- Bernoulli
@lru_cache(maxsize=None)
def bernoulli_numbers(n: int) -> tuple:
    """B_0..B_n with B_1 = -1/2 (sum_{k=0}^{m} C(m+1, k) B_k = 0, m >= 1)."""
    B = [Fraction(1)]
    for m in range(1, n + 1):
        s = sum(Fraction(math.comb(m + 1, k)) * B[k] for k in range(m))
        B.append(-s / (m + 1))
    return tuple(B)


def bernoulli_poly(n: int, x: Fraction) -> Fraction:
    B = bernoulli_numbers(n)
    return sum(Fraction(math.comb(n, k)) * B[k] * x ** (n - k) for k in range(n + 1))


def alpert_moments(p: int, kappa: int) -> list:
    """c_m = B_{m+1}(kappa) / (m + 1), m = 0..2p-1 (exact)."""
    return [bernoulli_poly(m + 1, Fraction(kappa)) / (m + 1) for m in range(2 * p)]


def _solve_exact(A, b):
    n = len(b)
    M = [list(row) + [bb] for row, bb in zip(A, b)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [v / pv for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * c for a, c in zip(M[r], M[col])]
    return [M[i][n] for i in range(n)]


@lru_cache(maxsize=None)
def alpert_rule(p: int, kappa: int, digits: int = 60):
    """Nodes x_1..x_p (ascending) and weights w_1..w_p of the one-sided
    endpoint correction of order 2p with kappa omitted regular nodes."""
    c = alpert_moments(p, kappa)
    # Prony: sum_i a_i c_{m+i} = -c_{m+p}, m = 0..p-1
    A = [[c[m + i] for i in range(p)] for m in range(p)]
    a = _solve_exact(A, [-c[m + p] for m in range(p)])
    coeffs = list(a) + [Fraction(1)]                       # ascending, monic
    guess = np.roots([float(v) for v in reversed(coeffs)])
    if np.max(np.abs(guess.imag)) > 1e-6:
        raise ValueError("Alpert moment system has complex nodes for p=%d kappa=%d" % (p, kappa))
    getcontext().prec = digits
    cd = [Decimal(v.numerator) / Decimal(v.denominator) for v in coeffs]

    def P(x):
        r = Decimal(0)
        for v in reversed(cd):
            r = r * x + v
        return r

    def dP(x):
        r = Decimal(0)
        for k in range(len(cd) - 1, 0, -1):
            r = r * x + cd[k] * k
        return r

    nodes = []
    for g in sorted(guess.real):
        x = Decimal(repr(float(g)))
        for _ in range(200):
            dx = P(x) / dP(x)
            x -= dx
            if abs(dx) < Decimal(10) ** (-(digits - 5)):
                break
        nodes.append(x)
    # weights: sum_k w_k x_k^m = c_m, m = 0..p-1 (Gaussian elimination in Decimal)
    cdm = [Decimal(v.numerator) / Decimal(v.denominator) for v in c]
    V = [[x ** m for x in nodes] + [cdm[m]] for m in range(p)]
    for col in range(p):
        piv = max(range(col, p), key=lambda r: abs(V[r][col]))
        V[col], V[piv] = V[piv], V[col]
        pv = V[col][col]
        V[col] = [v / pv for v in V[col]]
        for r in range(p):
            if r != col:
                f = V[r][col]
                V[r] = [x - f * y for x, y in zip(V[r], V[col])]
    w = [V[k][p] for k in range(p)]
    return tuple(float(x) for x in nodes), tuple(float(v) for v in w)


def alpert_residuals(p: int, kappa: int) -> float:
    """max_m |sum_k w_k x_k^m - c_m| / max(1, |c_m|) in double (a check)."""
    x, w = alpert_rule(p, kappa)
    c = alpert_moments(p, kappa)
    x = np.array(x)
    w = np.array(w)
    return max(abs(float(np.sum(w * x ** m)) - float(c[m])) / max(1.0, abs(float(c[m]))) for m in range(2 * p))


KAPPA_FOR_P = {8: 7}      # the paper's choice for p = 8 (Sec. 7, Example 2)


# ----------------------------------------------------------------- Gamma rule
def choose_H(eps: float, vnorm: float, phimax: float, d: int, eps_m: float = EPS_M) -> float:
    """Remark Hchoice; eps_m is the machine epsilon of the arithmetic that
    evaluates the contour sums (FP64 by default, 2^-23 for FP32 sums)."""
    return math.log(eps / ((1.0 + vnorm) * eps_m)) / (2.0 * d * (1.0 + phimax))


class GammaRule:
    """Nodes zeta_k (complex) and weights w_k on Gamma_K for one dimension, in
    the block order E1, A1, C, A3, E3 (Sec. 3.4)."""

    def __init__(self, M: int, H: float, NE: int, p: int = 8, kappa: int = None, q: int = 10, n_r: int = 1):
        self.M, self.H, self.NE, self.p, self.q, self.n_r = M, H, NE, p, q, n_r
        self.kappa = KAPPA_FOR_P.get(p, p) if kappa is None else kappa
        self.K = H + math.pi * M / 2.0
        self.h = (self.K - H) / (NE + 2 * self.kappa - 1)
        self.nu = 2 * (NE + 2 * self.kappa - 1)
        xa, wa = alpert_rule(p, self.kappa)
        h = self.h
        # Gamma_3
        tau_e3 = H + self.kappa * h + h * np.arange(NE)
        z_e3 = tau_e3 - 1j * H
        w_e3 = np.full(NE, h, dtype=np.complex128)
        z_a3 = H + np.array(xa) * h - 1j * H
        w_a3 = h * np.array(wa, dtype=np.complex128)
        # Gamma_1 by reflection
        z_e1 = -z_e3[::-1]
        w_e1 = w_e3[::-1].copy()
        z_a1 = -z_a3[::-1]
        w_a1 = w_a3[::-1].copy()
        # Gamma_2: composite Gauss-Legendre on dyadic panels, zeta = (1 - i) tau
        xg, wg = np.polynomial.legendre.leggauss(q)
        if n_r == 0:
            edges = [-H, H]
        else:
            pos = [0.0] + [H / 2.0 ** (n_r - k) for k in range(1, n_r + 1)]
            edges = [-e for e in reversed(pos[1:])] + pos
        tau_c, w_c = [], []
        for a, b in zip(edges[:-1], edges[1:]):
            tau_c.append(0.5 * (b - a) * xg + 0.5 * (a + b))
            w_c.append((1 - 1j) * 0.5 * (b - a) * wg)
        tau_c = np.concatenate(tau_c)
        self.tau_c = tau_c
        z_c = (1 - 1j) * tau_c
        w_c = np.concatenate(w_c)
        self.blocks = {"E1": (z_e1, w_e1), "A1": (z_a1, w_a1), "C": (z_c, w_c), "A3": (z_a3, w_a3),
                       "E3": (z_e3, w_e3)}
        self.zeta = np.concatenate([z_e1, z_a1, z_c, z_a3, z_e3])
        self.w = np.concatenate([w_e1, w_a1, w_c, w_a3, w_e3])
        self.N = self.zeta.size

    @staticmethod
    def for_nu(M: int, nu: int, H: float, p: int = 8, q: int = 10, n_r: int = 1, kappa: int = None):
        k = KAPPA_FOR_P.get(p, p) if kappa is None else kappa
        NE = nu // 2 - 2 * k + 1
        if NE <= M // 2:
            raise ValueError("need NE > M/2 (Sec. 4)")
        return GammaRule(M, H, NE, p=p, kappa=k, q=q, n_r=n_r)
