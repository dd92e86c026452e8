"""Pins for the iterative FP64 oracle (restarted GMRES on the matrix-free Eq. 7
operator, preconditioned by the per-mode free propagator) and for the mode-space
incident source of Eq. 7.

The iterative oracle is what the full-size GPU parity rests on, so it is pinned
here against routes that share none of its steps: the sparse LU of the assembled
matrix (``transport.solve``, ``operator.free_inverse``), the flat-potential
closed form (T = identity), and, for the source, the real-space construction of
b with the dense Eq. 8 block."""
import numpy as np
import pytest

import iobm_synth as S
from oracle import iterative, modes, operator, transport


def kb_junction(nf=4):
    return S.small_wire(nx=12, ny=12, nz=26, h=0.5, natom=2, spacing=3.4, depth=0.7, width=0.9,
                        rs=1.6, kb_kinds=S.SP, nf=nf, seed=77)


@pytest.mark.parametrize("nf,kappa", [(4, (0.0, 0.0)), (1, (0.0, 0.0)), (4, (0.21, -0.13))])
def test_free_propagator_equals_sparse_lu(nf, kappa):
    # the banded per-mode solve of (E - T - H~) against the LU of the assembled matrix
    jn = S.small_wire(nx=10, ny=9, nz=18, h=0.55, natom=1, depth=0.4, rs=1.5, nf=nf, seed=3)
    E = jn.e_fermi - 0.03
    md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, nf, E, kappa=kappa)
    r = S.random_field((jn.nz, jn.ny, jn.nx), 11)
    z = iterative.free_propagator_modes(jn, E, md, r)
    ref = operator.free_inverse(jn, E, md, r)
    assert np.max(np.abs(z - ref)) < 1e-11 * np.max(np.abs(ref))


def test_banded_systems_are_the_potential_free_operator():
    # A_free z computed by apply_A with V = 0 and no projectors reproduces r
    jn = S.small_wire(nx=8, ny=8, nz=16, h=0.6, natom=1, depth=0.5, rs=1.5, nf=4, seed=4)
    E = jn.e_fermi + 0.02
    md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, 4, E)
    flat = jn.copy_with(V=np.zeros_like(jn.V), projectors=[])
    r = S.random_field((jn.nz, jn.ny, jn.nx), 5)
    z = iterative.free_propagator_modes(jn, E, md, r)
    back = operator.apply_A(flat, E, md, z)
    assert np.max(np.abs(back - r)) < 1e-11 * np.max(np.abs(r))


@pytest.mark.parametrize("side", ["L", "R"])
def test_gmres_equals_sparse_lu(side):
    jn = kb_junction()
    E = jn.e_fermi
    ref = transport.solve(jn, E, side=side)
    it = iterative.solve_gmres(jn, E, side=side, tol=1e-12)
    assert np.all(it.residuals <= 1e-12)
    assert it.n_open == ref.n_open >= 3
    assert np.max(np.abs(it.t - ref.t)) < 1e-9
    assert np.max(np.abs(it.r - ref.r)) < 1e-9
    assert np.max(np.abs(it.T - ref.T)) < 1e-9
    assert abs(it.G - ref.G) < 1e-9
    assert np.max(np.abs(it.psi - ref.psi)) < 1e-9 * np.max(np.abs(ref.psi))


def test_gmres_flat_potential_integer_conductance():
    jn = S.small_wire(nx=12, ny=10, nz=20, h=0.6, natom=1, depth=0.0, rs=1.5, nf=4)
    jn = jn.copy_with(V=np.zeros_like(jn.V))
    it = iterative.solve_gmres(jn, jn.e_fermi)
    n = it.n_open
    assert n >= 3
    assert np.max(np.abs(it.T - np.eye(n))) < 1e-10
    assert abs(it.G - n) < 1e-10
    # the free propagator is the exact inverse here: one preconditioned step suffices
    assert np.all(it.gmres_iterations <= 3)


@pytest.mark.parametrize("nf", [1, 4])
def test_incident_source_mode_equals_eq19_of_real_space_source(nf):
    # b~[d] of Eq. 7 in mode space against the lateral transform (Eq. 19, explicit
    # sums) of the real-space source built from the electrode couplings and the dense
    # Eq. 8 self-energy block, for every open channel of both ends
    jn = S.small_wire(nx=10, ny=8, nz=3 * nf + 4, h=0.55, natom=1, depth=0.3, rs=1.3, nf=nf,
                      seed=21)
    E = jn.e_fermi
    md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, nf, E)
    F = modes.lateral_phase(jn.nx, jn.ny, jn.hx, jn.hy, md)
    nxy = jn.nx * jn.ny
    assert len(md.open_modes) >= 3
    for m in md.open_modes:
        bt = modes.incident_source_mode(md, m)
        for side in ("L", "R"):
            b = transport.source_vector(jn, md, m, side).reshape(jn.nz, nxy)
            planes = operator.end_planes(jn, side)
            ft = (F @ b[planes].T) / nxy           # [mode][depth]
            assert np.max(np.abs(ft[m] - bt)) < 1e-11 * np.max(np.abs(bt))
            others = np.delete(ft, m, axis=0)
            assert np.max(np.abs(others)) < 1e-11 * np.max(np.abs(bt))


def test_incident_source_mode_nf1_closed_form():
    # N_f = 1: b~ = (i / h_z^2) sin(k h_z) (Eq. 7 with Eq. 18-2)
    jn = S.small_wire(nx=9, ny=7, nz=8, h=0.5, natom=1, depth=0.0, rs=1.3, nf=1)
    md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, 1, jn.e_fermi)
    for m in md.open_modes:
        kh = np.angle(md.lam[m, md.prop[m]])
        bt = modes.incident_source_mode(md, m)
        assert abs(bt[0] - 1j * np.sin(kh) / jn.hz ** 2) < 1e-12 / jn.hz ** 2
