"""phi(t) = int_0^t A(s) ds (eq. phi), oracle side (test infrastructure only).

phi enters every phase factor of the recurrence (eqs. uhatkinteq, uhatkrecur).
Two independent evaluations are provided:
  * ``phi_pulse``: closed form for A(t) = A0 sin^2(pi t/Tp) sin(omega t) e,
    obtained by writing sin^2 = (1 - cos(2 pi t/Tp))/2 and integrating the
    three resulting sines exactly;
  * ``phi_quadrature``: composite Gauss-Legendre for any callable A.
"""
from __future__ import annotations

import math

import numpy as np


def _int_sin(a: float, t):
    """int_0^t sin(a s) ds = (1 - cos(a t))/a = 2 sin^2(a t/2)/a (0 if a = 0)."""
    if a == 0.0:
        return np.zeros_like(t)
    return 2.0 * np.sin(0.5 * a * t) ** 2 / a


def phi_pulse(t, A0: float, omega: float, T_pulse: float, direction) -> np.ndarray:
    """Closed-form phi for the sin^2 pulse; returns shape t.shape + (d,).

    A0 sin^2(pi t/Tp) sin(w t) = (A0/2)[sin(w t) - (sin((w+W)t) + sin((w-W)t))/2]
    with W = 2 pi / Tp, integrated term by term.
    """
    t = np.asarray(t, dtype=np.float64)
    W = 2.0 * math.pi / T_pulse
    val = 0.5 * A0 * (_int_sin(omega, t)
                      - 0.5 * (_int_sin(omega + W, t) + _int_sin(omega - W, t)))
    return np.multiply.outer(val, np.asarray(direction, dtype=np.float64))


def gauss_legendre(q: int):
    """q-point Gauss-Legendre nodes/weights on [-1,1] (numpy's Golub-Welsch)."""
    return np.polynomial.legendre.leggauss(q)


def phi_quadrature(A, t: float, d: int, panels_per_unit: int = 64, q: int = 20) -> np.ndarray:
    """phi(t) for a general vectorised A(t) -> (..., d) by composite Gauss-Legendre."""
    if t == 0.0:
        return np.zeros(d)
    npan = max(1, int(math.ceil(abs(t) * panels_per_unit)))
    x, w = gauss_legendre(q)
    edges = np.linspace(0.0, t, npan + 1)
    acc = np.zeros(d)
    for a, b in zip(edges[:-1], edges[1:]):
        s = 0.5 * (b - a) * x + 0.5 * (a + b)
        vals = np.asarray(A(s)).reshape(q, d)
        acc += 0.5 * (b - a) * (w @ vals)
    return acc


def phi_callable(pulse, d: int):
    """phi as a function of scalar t for a synth.Pulse (closed form) or None (A = 0)."""
    if pulse is None:
        return lambda t: np.zeros(d)
    return lambda t: phi_pulse(t, pulse.A0, pulse.omega, pulse.T_pulse, pulse.direction).reshape(d)
