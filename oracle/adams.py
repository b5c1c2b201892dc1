"""Implicit Adams quadrature weights (oracle; test infrastructure only).

Sec. 2.2 ("Higher-order time discretizations"): interpolate g at the n
points t - j dt, j = 0..n-1, by a polynomial of degree n-1 found from a
Vandermonde system, integrate it over [t - dt, t], and read off
int_{t-dt}^t g ~= dt * sum_j mu_j g(t - j dt).  With s = t - theta dt the
conditions are sum_j mu_j j^m = int_0^1 theta^m dtheta = 1/(m+1),
m = 0..n-1.  Solved here exactly in rational arithmetic.
Table 1 of the paper lists the n = 8 result; the trapezoidal rule is n = 2.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def weights_exact(n: int) -> list:
    """mu_0..mu_{n-1} as Fractions from the Vandermonde system (Sec. 2.2)."""
    if n < 1:
        raise ValueError("order must be >= 1")
    # Row m: sum_j j^m mu_j = 1/(m+1).  Gauss-Jordan elimination over Q.
    A = [[Fraction(j) ** m for j in range(n)] + [Fraction(1, m + 1)] for m in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        p = A[col][col]
        A[col] = [v / p for v in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [a - f * b for a, b in zip(A[r], A[col])]
    return [A[j][n] for j in range(n)]


def weights(n: int) -> np.ndarray:
    """mu_j as float64 (each the correctly rounded value of the exact rational)."""
    return np.array([float(w) for w in weights_exact(n)], dtype=np.float64)
