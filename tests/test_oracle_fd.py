"""Pins for the oracle's finite-difference weights (Eq. 1)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle.fd import second_derivative_weights, second_derivative_weights_exact


def test_nf1_matches_appendix():
    # Appendix, below Eq. A-03: c_0 = -2/h^2, c_{+-1} = 1/h^2
    assert second_derivative_weights_exact(1) == [Fraction(-2), Fraction(1)]


def test_nf4_matches_textbook_eighth_order():
    # Standard eighth-order central weights for f'' (Fornberg, Math. Comp. 51, 699 (1988)),
    # the "9-point" stencil of the 16x16x64 wire workload.
    assert second_derivative_weights_exact(4) == [
        Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315), Fraction(-1, 560)]


@pytest.mark.parametrize("nf", [1, 2, 3, 4, 5])
def test_exact_on_polynomials(nf):
    w = second_derivative_weights_exact(nf)
    x0 = Fraction(3, 7)
    for deg in range(0, 2 * nf + 2):
        approx = sum(w[abs(n)] * (x0 + n) ** deg for n in range(-nf, nf + 1))
        exact = deg * (deg - 1) * x0 ** (deg - 2) if deg >= 2 else 0
        assert approx == exact, (nf, deg)
    # and not exact one degree higher (the order is exactly 2 N_f)
    deg = 2 * nf + 2
    approx = sum(w[abs(n)] * (x0 + n) ** deg for n in range(-nf, nf + 1))
    assert approx != deg * (deg - 1) * x0 ** (deg - 2)


def test_symbol_monotone_nf4():
    # one propagating pair per lateral mode needs a monotone 1D dispersion on [0, pi]
    w = second_derivative_weights(4)
    th = np.linspace(0, np.pi, 2001)
    eps = -0.5 * (w[0] + 2 * sum(w[n] * np.cos(n * th) for n in range(1, 5)))
    assert np.all(np.diff(eps) > 0)
