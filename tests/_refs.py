"""Independent reference solutions used to pin the oracle (test helpers).

Nothing here imports the oracle.  The references are
  * the exact free-particle solution with advection for a trigonometric
    polynomial u0 (eq. uhatkinteq with V = 0),
  * the pseudo-spectral semi-discrete system i u' = F^{-1} diag(|k|^2 - k.A(t)) F u + V u
    integrated by scipy's DOP853 at tight tolerance (numpy.fft for F), and
  * the dense propagator exp(-i H T) by a Hermitian eigendecomposition
    (numpy.linalg.eigh) for time-independent V and A = 0.
The scheme converges to the last two as dt -> 0 (Sec. 2.2), at the Adams order.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp


def fft_wavenumbers(M: int) -> np.ndarray:
    """numpy's ordering; index M/2 carries k = -M/2 (the paper's truncation)."""
    return np.fft.fftfreq(M, d=1.0 / M)


def grid(M: int) -> np.ndarray:
    return -math.pi + 2.0 * math.pi * np.arange(M) / M


def exact_free(coeffs: dict, shape, t: float, phi_t) -> np.ndarray:
    """u(x,t) = sum_k c_k exp(i k.x - i |k|^2 t + i k.phi(t)) on the grid."""
    grids = np.meshgrid(*[grid(M) for M in shape], indexing="ij")
    u = np.zeros(shape, dtype=np.complex128)
    for k, c in coeffs.items():
        arg = sum(kk * g for kk, g in zip(k, grids)) - sum(kk * kk for kk in k) * t \
            + sum(kk * p for kk, p in zip(k, phi_t))
        u += c * (np.cos(arg) + 1j * np.sin(arg))
    return u


def ode_reference(shape, u0, V0, vfac, A, T: float, rtol: float = 1e-13, atol: float = 1e-14):
    """Pseudo-spectral semi-discrete solution at time T (DOP853)."""
    shape = tuple(shape)
    d = len(shape)
    ks = np.meshgrid(*[fft_wavenumbers(M) for M in shape], indexing="ij")
    ksq = sum(k * k for k in ks)
    n = int(np.prod(shape))

    def rhs(t, y):
        u = (y[:n] + 1j * y[n:]).reshape(shape)
        a = np.zeros(d) if A is None else np.asarray(A(t), dtype=np.float64).reshape(d)
        sym = ksq - sum(ks[i] * a[i] for i in range(d))
        du = -1j * (np.fft.ifftn(sym * np.fft.fftn(u)) + float(vfac(t)) * V0 * u)
        du = du.reshape(-1)
        return np.concatenate([du.real, du.imag])

    y0 = np.concatenate([u0.reshape(-1).real, u0.reshape(-1).imag])
    sol = solve_ivp(rhs, (0.0, T), y0, method="DOP853", rtol=rtol, atol=atol)
    assert sol.success
    y = sol.y[:, -1]
    return (y[:n] + 1j * y[n:]).reshape(shape)


def dense_propagator_1d(u0, V0, T: float):
    """exp(-i H T) u0 with H = F^{-1} diag(k^2) F + diag(V0), via eigh."""
    M = u0.shape[0]
    k = fft_wavenumbers(M)
    I = np.eye(M)
    K = np.fft.ifft(k[:, None] ** 2 * np.fft.fft(I, axis=0), axis=0)
    H = K + np.diag(V0)
    H = 0.5 * (H + H.conj().T)
    w, Q = np.linalg.eigh(H)
    return Q @ (np.exp(-1j * w * T) * (Q.conj().T @ u0))
