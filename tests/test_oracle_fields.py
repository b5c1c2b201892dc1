"""Pins for the oracle's phi(t) = int_0^t A(s) ds (eq. phi)."""
import math

import numpy as np
import pytest

from oracle import fields
from synth import Pulse


@pytest.mark.parametrize("pulse", [
    Pulse(2.0, 10.0, 2.0, (1.0, 0.0)),
    Pulse(3.0, 10.0, 1.0, (1.0,)),
    Pulse(1.5, math.pi, 2.0, (0.6, 0.8)),      # omega equal to 2 pi / Tp: degenerate term
])
def test_closed_form_matches_gauss_legendre(pulse):
    d = len(pulse.direction)
    for t in (0.0, 1e-3, 0.37, 1.0, 1.9999):
        cf = fields.phi_pulse(t, pulse.A0, pulse.omega, pulse.T_pulse, pulse.direction).reshape(d)
        gl = fields.phi_quadrature(pulse.A, t, d)
        assert np.allclose(cf, gl, rtol=0, atol=2e-15), (t, cf, gl)


def test_derivative_is_A():
    p = Pulse(2.0, 10.0, 2.0, (1.0, 0.0))
    for t in (0.2, 0.9, 1.7):
        e = 1e-5
        dphi = (fields.phi_pulse(t + e, p.A0, p.omega, p.T_pulse, p.direction)
                - fields.phi_pulse(t - e, p.A0, p.omega, p.T_pulse, p.direction)) / (2 * e)
        assert np.allclose(dphi, p.A(t), atol=1e-8)


def test_zero_and_constant_field():
    assert np.all(fields.phi_callable(None, 2)(0.7) == 0.0)
    A = lambda s: np.multiply.outer(np.ones_like(np.asarray(s)), np.array([1.25, -0.5]))
    assert np.allclose(fields.phi_quadrature(A, 0.8, 2), [1.0, -0.4], atol=1e-15)
