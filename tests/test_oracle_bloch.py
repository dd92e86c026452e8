"""Pins for the oracle at a lateral Bloch vector kappa != 0 (Eq. 8: modes G_nu + kappa,
psi(r + L) = exp(i kappa L) psi(r)).  The operator is then no longer complex symmetric:
A(kappa)^T = A(-kappa)."""
import math

import numpy as np
import pytest

import iobm_synth as S
from oracle import modes, operator, transport
from oracle.fd import second_derivative_weights
from test_oracle_transport import transfer_T_nf1


def kappa_of(jn, fx, fy):
    """kappa as fractions of the first Brillouin-zone half-width pi / L."""
    return (fx * math.pi / (jn.nx * jn.hx), fy * math.pi / (jn.ny * jn.hy))


def flat_junction(nf, nx=12, ny=10, nz=14, h=0.6, rs=1.5):
    jn = S.small_wire(nx=nx, ny=ny, nz=nz, h=h, natom=1, depth=0.0, rs=rs, nf=nf)
    return jn.copy_with(V=np.zeros_like(jn.V))


def kb_junction(nf=4):
    return S.small_wire(nx=12, ny=12, nz=26, h=0.5, natom=2, spacing=3.4, depth=0.7, width=0.9,
                        rs=1.6, kb_kinds=S.SP, nf=nf, seed=77)


def test_kappa_zero_is_the_periodic_solution():
    jn = kb_junction(4)
    E = jn.e_fermi
    a = transport.solve(jn, E)
    b = transport.solve(jn, E, kappa=(0.0, 0.0))
    assert np.array_equal(a.T, b.T) and np.array_equal(a.R, b.R)


def test_transpose_is_minus_kappa():
    # complex symmetry is lost, but A(kappa)^T = A(-kappa): the Bloch phases of the
    # wrapped couplings conjugate, and Sigma~ depends on |G + kappa| only
    jn = S.small_wire(nx=8, ny=6, nz=12, h=0.6, natom=1, depth=0.5, rs=1.5, nf=4)
    E = jn.e_fermi
    k = kappa_of(jn, 0.37, -0.21)
    A = operator.assemble_A_local(jn, E, transport.modes_for(jn, E, k))
    Am = operator.assemble_A_local(jn, E, transport.modes_for(jn, E, (-k[0], -k[1])))
    assert abs(A - A.T).max() > 1e-3                  # not symmetric
    assert abs(A.T - Am).max() < 1e-12 * abs(A).max()


@pytest.mark.parametrize("nf", [1, 4])
@pytest.mark.parametrize("fx,fy", [(0.3, 0.0), (0.45, -0.7)])
def test_flat_potential_integer_conductance(nf, fx, fy):
    jn = flat_junction(nf)
    k = kappa_of(jn, fx, fy)
    sol = transport.solve(jn, jn.e_fermi, kappa=k)
    assert sol.n_open >= 2
    assert np.max(np.abs(sol.T - np.eye(sol.n_open))) < 1e-10
    assert np.max(np.abs(sol.R)) < 1e-10
    assert abs(sol.G - sol.n_open) < 1e-10


def test_open_channel_count_at_kappa():
    # modes whose z band holds E: 0 < E - eps_perp(G + kappa) < band top, with the
    # lateral dispersion written out here from the FD weights
    jn = flat_junction(4, nx=16, ny=14, h=0.5, rs=1.3)
    w = second_derivative_weights(4)
    for fx, fy in [(0.0, 0.0), (0.3, 0.6), (-0.8, 0.2)]:
        k = kappa_of(jn, fx, fy)
        E = jn.e_fermi

        def eps1(n, h, kap):
            G = 2 * math.pi * (np.arange(n) - n // 2) / (n * h) + kap
            return -0.5 * (w[0] + 2 * sum(w[j] * np.cos(j * G * h) for j in range(1, 5))) / h ** 2

        ex, ey = eps1(jn.nx, jn.hx, k[0]), eps1(jn.ny, jn.hy, k[1])
        top = -0.5 * (w[0] + 2 * sum(w[j] * (-1) ** j for j in range(1, 5))) / jn.hz ** 2
        dE = E - (ey[:, None] + ex[None, :])
        expect = int(np.sum((dE > 0) & (dE < top)))
        got = modes.count_open_channels(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, 4, E, kappa=k)
        assert got == expect


@pytest.mark.parametrize("nf", [1, 4])
def test_current_conservation_at_kappa(nf):
    jn = kb_junction(nf)
    sol = transport.solve(jn, jn.e_fermi, kappa=kappa_of(jn, 0.41, -0.27))
    assert sol.n_open >= 3
    per_in = sol.T.sum(axis=0) + sol.R.sum(axis=0)
    assert np.max(np.abs(per_in - 1.0)) < 1e-10


def test_reciprocity_kappa_to_minus_kappa():
    # time reversal maps (nu, kappa) to (-nu, -kappa): T^{L->R}(kappa)[o, i] equals
    # T^{R->L}(-kappa)[i~, o~] with ~ the reversed mode
    jn = kb_junction(4)
    E = jn.e_fermi - 0.02
    k = kappa_of(jn, 0.33, 0.52)
    L = transport.solve(jn, E, side="L", kappa=k)
    R = transport.solve(jn, E, side="R", kappa=(-k[0], -k[1]))
    nu_R = [tuple(R.md.nu[m]) for m in R.open_modes]

    def rev(a, n):
        return -a if -a in range(-(n // 2), n - n // 2) else a

    flip = [nu_R.index((rev(a, jn.nx), rev(b, jn.ny))) for a, b in (tuple(L.md.nu[m]) for m in L.open_modes)]
    assert L.n_open == R.n_open
    for o in range(L.n_open):
        for i in range(L.n_open):
            assert abs(L.T[o, i] - R.T[flip[i], flip[o]]) < 1e-10
    assert abs(L.G - R.G) < 1e-10


def test_reciprocal_lattice_shift():
    # kappa and kappa + 2 pi / L_x describe the same Bloch waves: same conductance
    jn = kb_junction(4)
    E = jn.e_fermi
    k = kappa_of(jn, 0.3, 0.1)
    k2 = (k[0] + 2 * math.pi / (jn.nx * jn.hx), k[1])
    assert abs(transport.conductance(jn, E, k) - transport.conductance(jn, E, k2)) < 1e-9


def test_uniform_vz_transfer_matrix_at_kappa():
    # laterally uniform V(z): modes decouple; each is the 1D chain at E - eps_perp(G + kappa)
    nx, ny, nz, h = 10, 9, 30, 0.5
    jn = S.small_wire(nx=nx, ny=ny, nz=nz, h=h, natom=1, depth=0.0, rs=1.2, nf=1)
    z = np.arange(nz) * h
    Vz = 0.35 * np.exp(-((z - 7.0) / 1.3) ** 2) - 0.2 * np.exp(-((z - 9.5) / 0.8) ** 2)
    jn = jn.copy_with(V=np.broadcast_to(Vz[:, None, None], (nz, ny, nx)).copy())
    E = jn.e_fermi
    sol = transport.solve(jn, E, kappa=kappa_of(jn, 0.6, -0.35))
    md = sol.md
    assert sol.n_open >= 2
    for i, m in enumerate(sol.open_modes):
        Tm, Rm = transfer_T_nf1(Vz, E - md.eps_perp[m], h)
        assert abs(sol.T[i, i] - Tm) < 1e-10
        assert abs(sol.R[i, i] - Rm) < 1e-10


def test_matrix_free_operator_at_kappa():
    # the matrix-free operator (Bloch-wrapped shifts, explicit Eq. 19 sums) equals the
    # assembled one, and the FFT route of the self-energy equals the explicit sums
    jn = S.small_wire(nx=9, ny=8, nz=12, h=0.6, natom=1, depth=0.5, rs=1.5, nf=4,
                      kb_kinds=S.SP, kb_radius=1.2, kb_width=0.5, seed=3)
    E = jn.e_fermi
    md = transport.modes_for(jn, E, kappa_of(jn, -0.4, 0.75))
    rng = np.random.default_rng(5)
    psi = rng.standard_normal((jn.nz, jn.ny, jn.nx)) + 1j * rng.standard_normal((jn.nz, jn.ny, jn.nx))
    A = operator.assemble_A_local(jn, E, md)
    P, cpl, dv = operator.kb_factors(jn)
    ref = A @ psi.reshape(-1) - dv * (P @ (cpl * (P.T @ psi.reshape(-1))))
    got = operator.apply_A(jn, E, md, psi).reshape(-1)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    planes = psi[:4].reshape(4, -1)
    explicit = operator._sigma_apply_end(jn, md, planes)
    fft = operator._sigma_apply_end_fft(jn, md, planes)
    assert np.max(np.abs(explicit - fft)) < 1e-12 * np.max(np.abs(explicit))


def test_gradient_at_kappa_matches_finite_differences():
    jn = S.small_wire(nx=8, ny=8, nz=20, h=0.6, natom=2, spacing=3.0, depth=0.6, width=0.9,
                      rs=1.5, kb_kinds=S.SP, kb_radius=1.2, kb_width=0.5, seed=11, nf=4)
    E = jn.e_fermi
    k = kappa_of(jn, 0.35, -0.2)
    g = transport.grad_V(jn, E, kappa=k)
    rng = np.random.default_rng(2)
    dv = 1e-5
    for _ in range(3):
        p = (rng.integers(5, jn.nz - 5), rng.integers(0, jn.ny), rng.integers(0, jn.nx))
        Vp = jn.V.copy()
        Vp[p] += dv
        Vm = jn.V.copy()
        Vm[p] -= dv
        fd = (transport.conductance(jn.copy_with(V=Vp), E, k)
              - transport.conductance(jn.copy_with(V=Vm), E, k)) / (2 * dv)
        assert abs(g[p] - fd) < 1e-6 * max(1.0, abs(fd))
