"""Central finite-difference weights for the second derivative (Eq. 1).

Eq. 1 writes d^2 psi/dr^2 as sum_{n=-N_f}^{N_f} c_{mu,n} psi(r + n h_mu e_mu) and
takes the weights from the literature; for N_f = 1 the paper works them out
(Appendix, below Eq. A-03): c_0 = -2/h^2, c_{+-1} = 1/h^2.

Here the dimensionless weights w_n (c_{mu,n} = w_|n| / h_mu^2) are the unique
symmetric solution of the Taylor conditions

    sum_{n=-N_f}^{N_f} w_|n| n^(2m) = 2 * [m == 1],   m = 0 .. N_f,

solved exactly in rational arithmetic.

Pinned by: N_f = 1 against the Appendix values; N_f = 4 against the
textbook eighth-order weights (-205/72, 8/5, -1/5, 8/315, -1/560); exactness
on polynomials of degree <= 2 N_f + 1 (tests/test_oracle_fd.py).
"""
from __future__ import annotations

from fractions import Fraction
from typing import List

import numpy as np


def second_derivative_weights_exact(nf: int) -> List[Fraction]:
    """Exact weights [w_0, w_1, ..., w_nf] (Eq. 1, dimensionless)."""
    if nf < 1:
        raise ValueError("N_f must be >= 1")
    n_unk = nf + 1
    # rows m = 0..nf, columns w_0..w_nf
    M = [[Fraction(0)] * n_unk for _ in range(n_unk)]
    rhs = [Fraction(0)] * n_unk
    for m in range(n_unk):
        M[m][0] = Fraction(1) if m == 0 else Fraction(0)
        for n in range(1, nf + 1):
            M[m][n] = Fraction(2 * n ** (2 * m))
        rhs[m] = Fraction(2) if m == 1 else Fraction(0)
    # Gauss-Jordan elimination in exact arithmetic
    for col in range(n_unk):
        piv = next(r for r in range(col, n_unk) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        rhs[col], rhs[piv] = rhs[piv], rhs[col]
        inv = 1 / M[col][col]
        M[col] = [a * inv for a in M[col]]
        rhs[col] *= inv
        for r in range(n_unk):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * b for a, b in zip(M[r], M[col])]
                rhs[r] -= f * rhs[col]
    return rhs


def second_derivative_weights(nf: int) -> np.ndarray:
    """Float64 weights [w_0 .. w_nf]; c_{mu,n} = w_|n| / h_mu^2 (Eq. 1)."""
    return np.array([float(w) for w in second_derivative_weights_exact(nf)])
