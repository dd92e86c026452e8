"""Pins for the oracle's operator, self-energy blocks and preconditioner."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import iobm_synth as S
from oracle import modes, operator

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small(nf=4, kb=True, nx=6, ny=5, nz=22):
    return S.small_wire(nx=nx, ny=ny, nz=nz, h=0.45, natom=2, spacing=2.6, depth=0.6, width=0.9,
                        rs=2.2, kb_kinds=S.SP if kb else None, nf=nf)


def full_matrix(jn, E, md):
    A = operator.assemble_A_local(jn, E, md)
    P, cpl, dv = operator.kb_factors(jn)
    if P.shape[1]:
        A = A - dv * P @ sp.diags(cpl) @ P.T
    return A.tocsr()


@pytest.mark.parametrize("nf", [1, 4])
def test_complex_symmetric(nf):
    jn = small(nf)
    E = jn.e_fermi
    md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, nf, E)
    A = full_matrix(jn, E, md)
    assert abs(A - A.T).max() < 1e-12 * abs(A).max()


@pytest.mark.parametrize("nf", [1, 4])
def test_matrix_free_equals_assembled(nf):
    jn = small(nf)
    E = jn.e_fermi + 0.01
    md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, nf, E)
    A = full_matrix(jn, E, md)
    x = S.random_field((jn.nz, jn.ny, jn.nx), 3)
    y1 = (A @ x.reshape(-1)).reshape(x.shape)
    y2 = operator.apply_A(jn, E, md, x)
    assert np.max(np.abs(y1 - y2)) < 1e-12 * np.max(np.abs(y1))


def test_dense_sigma_nf1_equals_appendix_green_function():
    # Eq. A-01 with Eq. A-10: Sigma_L = B^dagger G^r_L(z_-1, z_-1) B, B = -1/(2 h_z^2),
    # G^r_L = -(2 h_z^2 / N_xy) sum_nu exp(i G.(r_l - r_l')) exp(i k_z h_z)
    nx, ny, h = 4, 6, 0.5
    jn = S.small_wire(nx=nx, ny=ny, nz=8, h=h, natom=1, depth=0.0, nf=1)
    E = 0.31
    md = modes.mode_data(nx, ny, h, h, h, 1, E)
    Sd = operator.sigma_dense(jn, md)
    nxy = nx * ny
    B = -1.0 / (2 * h * h)
    for l in range(nxy):
        xl, yl = (l % nx) * h, (l // nx) * h
        for lp in range(nxy):
            xp, yp = (lp % nx) * h, (lp // nx) * h
            g = 0j
            for ny_ in modes.lateral_indices(ny):
                for nx_ in modes.lateral_indices(nx):
                    Gx, Gy = 2 * math.pi * nx_ / (nx * h), 2 * math.pi * ny_ / (ny * h)
                    chi = h * h * E - (1 - math.cos(Gx * h)) - (1 - math.cos(Gy * h)) - 1
                    kh = math.acos(-chi) if abs(chi) < 1 else 1j * math.acosh(-chi)
                    g += np.exp(1j * (Gx * (xl - xp) + Gy * (yl - yp))) * np.exp(1j * kh)
            g *= -2 * h * h / nxy
            assert abs(Sd[l, lp] - B * g * B) < 1e-13


def test_dense_sigma_equals_fourier_apply():
    # Eq. 8 (real-space dense sum) against Eqs. 18-1/19 (diagonal in lateral Fourier space)
    jn = small(4, kb=False)
    E = jn.e_fermi
    md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, 4, E)
    Sd = operator.sigma_dense(jn, md)
    v = S.random_field((4, jn.nx * jn.ny), 5)
    y1 = (Sd @ v.reshape(-1)).reshape(4, -1)
    y2 = operator._sigma_apply_end(jn, md, v)
    assert np.max(np.abs(y1 - y2)) < 1e-13 * np.max(np.abs(y1))


def _alphas():
    out = []
    with open(os.path.join(GOLDEN, "pcg_alpha.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                out.append(float(line.split()[0]))
    return out


def test_preconditioner_matrix_free_and_symmetric():
    jn = small(4, kb=False)
    x = S.random_field((jn.nz, jn.ny, jn.nx), 9)
    for a in _alphas():
        P = operator.P_matrix(jn, a)
        assert abs(P - P.T).max() == 0
        y1 = (P @ x.reshape(-1)).reshape(x.shape)
        assert np.max(np.abs(y1 - operator.apply_P(jn, a, x))) < 1e-14


def test_preconditioner_positive_for_paper_alphas():
    # Sec. III: alpha in {3.0, 2.4, 1.8}; with the six face neighbours P stays positive
    # definite for alpha > ln 6 (symbol 1 + 2 C_1 (cos tx + cos ty + cos tz) > 0).
    assert min(_alphas()) > math.log(6.0)
    jn = S.small_wire(nx=8, ny=8, nz=10, h=0.5, natom=1, depth=0.0)
    for a in _alphas():
        ev = np.linalg.eigvalsh(operator.P_matrix(jn, a).toarray())
        assert ev.min() > 0
    # the eight-corner reading of "(+-h_x, +-h_y, +-h_z)" would be indefinite at
    # alpha = 1.8 (symbol 1 - 8 exp(-1.8) < 0 at the zone corner), which is why
    # the face-neighbour reading is taken
    assert 1 - 8 * math.exp(-1.8) < 0
    # and just below ln 6 the face-neighbour P loses definiteness on a periodic grid
    c1 = math.exp(-(math.log(6.0) - 0.05))
    assert 1 - 6 * c1 < 0


@pytest.mark.parametrize("nx,ny,nf", [(12, 10, 4), (9, 8, 1), (16, 16, 2)])
def test_sigma_fft_route_matches_explicit_sums(nx, ny, nf):
    # the FFT route used for large planes gives the explicit Eq. 19 sums
    from oracle.operator import _sigma_apply_end_fft, lateral_phase
    jn = S.small_wire(nx=nx, ny=ny, nz=2 * nf + 3, h=0.5, natom=1, depth=0.0, rs=1.5, nf=nf)
    md = modes.mode_data(nx, ny, jn.hx, jn.hy, jn.hz, nf, jn.e_fermi)
    rng = np.random.default_rng(4)
    v = rng.standard_normal((nf, nx * ny)) + 1j * rng.standard_normal((nf, nx * ny))
    F = lateral_phase(nx, ny, jn.hx, jn.hy, md)
    ft = (F @ v.T) / (nx * ny)
    ref = (F.conj().T @ np.einsum("mde,me->md", md.sigma, ft)).T
    assert np.max(np.abs(_sigma_apply_end_fft(jn, md, v) - ref)) < 1e-12 * np.max(np.abs(ref))
