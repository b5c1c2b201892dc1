"""Pins for the oracle's implicit Adams weights (Sec. 2.2, Table 1)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import adams


def _read_table1(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "adams8_table1.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                j, num, den = line.split()
                rows.append((int(j), Fraction(int(num), int(den))))
    return [f for _, f in sorted(rows)]


def test_order8_matches_table1(golden_dir):
    """The Vandermonde solve reproduces the paper's Table 1 exactly."""
    table = _read_table1(golden_dir)
    assert adams.weights_exact(8) == table
    assert sum(table) == 1


def test_trapezoid_is_order2():
    """Sec. 2.2: the second-order method is the trapezoidal rule, mu_0 = mu_1 = 1/2."""
    assert adams.weights_exact(2) == [Fraction(1, 2), Fraction(1, 2)]


def test_order4_textbook():
    """Textbook 4th-order Adams-Moulton: (9, 19, -5, 1)/24."""
    assert adams.weights_exact(4) == [Fraction(9, 24), Fraction(19, 24), Fraction(-5, 24), Fraction(1, 24)]


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_weights_sum_to_one(n):
    assert sum(adams.weights_exact(n)) == 1


@pytest.mark.parametrize("n", [2, 4, 6, 8])
def test_local_order_on_smooth_integrand(n):
    """int_{t-h}^t e^s ds ~= h sum_j mu_j e^{t-jh}: local error O(h^{n+1})."""
    mu = adams.weights(n)
    t = 0.3
    errs = []
    for h in (0.1, 0.05):
        approx = h * sum(mu[j] * math.exp(t - j * h) for j in range(n))
        exact = math.exp(t) - math.exp(t - h)
        errs.append(abs(approx - exact))
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - (n + 1)) < 0.35, rate


def test_float_weights_correctly_rounded():
    w = adams.weights(8)
    for a, b in zip(w, adams.weights_exact(8)):
        assert a == float(b)
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=4e-16)
