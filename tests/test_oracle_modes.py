"""Pins for the oracle's electrode modes and self-energy (Eqs. 8-9, 17, 18-2, A-01..A-10)."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import modes
from oracle.fd import second_derivative_weights

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fermi(rs):
    return (9 * math.pi / 4) ** (2 / 3) / (2 * rs * rs)


def paper_kz(E, Gx, Gy, hx, hy, hz):
    """Eqs. 8.5 and 9 as printed (kappa = 0): returns k_z h_z (complex)."""
    chi = hz * hz * E - hz * hz / hx ** 2 * (1 - math.cos(Gx * hx)) \
        - hz * hz / hy ** 2 * (1 - math.cos(Gy * hy)) - 1
    if abs(chi) < 1:
        return math.acos(-chi)            # propagating, k_z > 0
    # evanescent: k_z = i arccosh(-chi)/h_z with -i k_z > 0 (chi < -1 here)
    assert -chi > 1
    return 1j * math.acosh(-chi)


@pytest.mark.parametrize("E", [0.05, 0.17, 0.6])
def test_sigma_nf1_equals_eq18_2(E):
    nx, ny, h = 6, 5, 0.45
    md = modes.mode_data(nx, ny, h, h, h, 1, E)
    for m in range(len(md.nu)):
        Gx = 2 * math.pi * md.nu[m, 0] / (nx * h)
        Gy = 2 * math.pi * md.nu[m, 1] / (ny * h)
        kh = paper_kz(E, Gx, Gy, h, h, h)
        expect = -1.0 / (2 * h * h) * np.exp(1j * kh)          # Eq. 18-2
        assert abs(md.sigma[m, 0, 0] - expect) < 1e-13 * abs(expect)
        # propagating exactly when |chi| < 1 (Eq. 8.5)
        assert (md.prop[m] >= 0) == (abs(np.imag(kh)) == 0)


def test_root_pair_product_is_one():
    # Eq. A-08: omega_1 omega_2 = 1 for the two roots of the N_f = 1 recurrence
    w = second_derivative_weights(1)
    for dE in (-3.0, -0.1, 0.2, 1.5):
        r = modes.z_roots(dE, w, 0.4)
        assert abs(r[0] * r[1] - 1) < 1e-13


def chain_surface_sigma(E_minus_eps, nf, hz, n_planes=6000):
    """Brute force (Eq. A-01): Sigma = K g K^T with g the Green's function of an
    explicit long electrode chain (planes e = 1..n_planes), g = (E - H_chain)^{-1}."""
    w = second_derivative_weights(nf)
    K = modes.coupling_matrix(w, hz)
    # banded H_chain of the 1D mode problem: -1/(2h^2) sum_n w_n shift^n (+eps on the diagonal)
    ab = np.zeros((2 * nf + 1, n_planes), dtype=complex)
    for n in range(-nf, nf + 1):
        ab[nf - n, :] = E_minus_eps + 0.5 * w[abs(n)] / hz ** 2 if n == 0 else 0.5 * w[abs(n)] / hz ** 2
    rhs = np.zeros((n_planes, nf), dtype=complex)
    rhs[:nf, :] = np.eye(nf)
    g = sla.solve_banded((nf, nf), ab, rhs)[:nf, :]
    return K @ g @ K.T


@pytest.mark.parametrize("nf", [1, 4])
@pytest.mark.parametrize("dE,eta", [(0.17, 0.05), (0.02, 0.08), (-0.3, 0.0), (-2.0, 0.0)])
def test_sigma_matches_explicit_chain(nf, dE, eta):
    hz = 0.4
    w = second_derivative_weights(nf)
    z = dE + 1j * eta
    roots = modes.z_roots(z, w, hz)
    lam = np.array(sorted([r for r in roots if abs(r) < 1], key=abs))
    assert len(lam) == nf
    sig = modes.sigma_mode(lam, modes.coupling_matrix(w, hz))
    brute = chain_surface_sigma(z, nf, hz)
    assert np.max(np.abs(sig - brute)) < 1e-10 * np.max(np.abs(brute))


@pytest.mark.parametrize("nf", [1, 4])
def test_retarded_limit(nf):
    # the velocity rule at real E is the eta -> 0+ limit of |lambda| < 1
    hz, dE = 0.4, 0.17
    w = second_derivative_weights(nf)
    lam, p, v = modes.right_going(modes.z_roots(dE, w, hz), w, hz)
    K = modes.coupling_matrix(w, hz)
    s0 = modes.sigma_mode(lam, K)
    for eta in (1e-5, 1e-6):
        r = modes.z_roots(dE + 1j * eta, w, hz)
        le = np.array([x for x in r if abs(x) < 1])
        # same ordering: match to the real-E roots
        le = np.array([le[np.argmin(np.abs(le - l))] for l in lam])
        assert np.max(np.abs(modes.sigma_mode(le, K) - s0)) < 50 * eta * np.max(np.abs(s0))
    assert p >= 0 and v > 0


def test_sigma_symmetric_and_dissipative():
    md = modes.mode_data(8, 8, 0.4, 0.4, 0.4, 4, 0.3)
    for m in range(len(md.nu)):
        s = md.sigma[m]
        assert np.max(np.abs(s - s.T)) < 1e-12 * np.max(np.abs(s))
        # retarded: -Im Sigma is positive semidefinite (zero for closed modes)
        ev = np.linalg.eigvalsh(0.5j * (s - s.conj().T))   # Gamma/2 = i(Sigma - Sigma^H)/2
        assert ev.min() > -1e-10 * np.max(np.abs(s))
        if md.prop[m] < 0:
            assert np.max(np.abs(s.imag)) < 1e-9 * np.max(np.abs(s))


def _golden_counts():
    rows = []
    with open(os.path.join(GOLDEN, "channel_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                lab, rs, L, N, nin, cite = line.split()
                rows.append((lab, float(rs), float(L), int(N), int(nin), cite))
    return rows


@pytest.mark.parametrize("nf", [1, 4])
def test_channel_count_ir_au(nf):
    # Sec. IV: N_in = 37 for the Ir and Au electrode cells
    for lab, rs, L, N, nin, cite in _golden_counts():
        if cite.endswith("unpinned"):
            continue
        h = L / N
        assert modes.count_open_channels(N, N, h, h, h, nf, fermi(rs)) == nin, lab


def test_channel_count_na_reading():
    # Sec. III prints N_in = 13 for the Na cell; free-electron counting gives 9
    # (5 modes with nu^2 <= 1 plus the 4 diagonal ones).  Recorded as a reading.
    (lab, rs, L, N, nin, cite), = [r for r in _golden_counts() if r[0] == "Na"]
    h = L / N
    assert nin == 13
    assert modes.count_open_channels(N, N, h, h, h, 4, fermi(rs)) == 9


def test_threshold_rejected():
    nx = ny = 8
    h = 0.4
    md = modes.mode_data(nx, ny, h, h, h, 4, 0.3)
    e_perp = np.unique(np.round(md.eps_perp, 12))
    with pytest.raises(modes.ThresholdError):
        modes.mode_data(nx, ny, h, h, h, 4, float(e_perp[1]) + 1e-12)


def test_eq19_matches_fft():
    # Eq. 19 with G_nu = 2 pi nu / L is numpy's forward FFT divided by N_xy
    rng = np.random.default_rng(0)
    nx, ny, h = 6, 10, 0.3
    md = modes.mode_data(nx, ny, h, h, h, 1, 0.2)
    plane = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    ft = modes.eq19_forward(nx, ny, h, h, md, plane)
    ref = np.fft.fft2(plane) / (nx * ny)
    for m in range(len(md.nu)):
        assert abs(ft[m] - ref[md.nu[m, 1] % ny, md.nu[m, 0] % nx]) < 1e-13
