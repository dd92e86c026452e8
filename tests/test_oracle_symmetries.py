"""Symmetry pins of the oracle: exact identities of the discrete transport problem
(Eqs. 1-8, 19, Landauer G of Sec. III) that a slip anywhere in the oracle's lateral
indexing, Bloch phases, end-plane handling or flux normalisation would break.

* lateral supercell: doubling the periodic cell along x at kappa = 0 folds the
  Bloch vectors 0 and pi / L_x of the original cell (the supercell's lateral modes
  2 pi m / (2 L_x) are the original G_nu for even m and G_nu + pi / L_x for odd m), so
  G_super(0) = G(0) + G(pi / L_x);
* x <-> y transposition of a non-square cell (nx != ny, h_x != h_y) leaves G unchanged;
* a lateral translation by whole grid steps multiplies each mode by a phase: T and R
  unchanged entry by entry;
* the mirror image z -> -z swaps the electrodes: T^{L->R} of the mirrored junction is
  T^{R->L} of the original, entry by entry;
* the supercell fold of the gradient: a perturbation with the original cell's period
  changes both folded problems, and the supercell's gradient is the same on both copies
  of the cell, so 2 dG_super/dV(r) = dG(0)/dV(r) + dG(pi / L_x)/dV(r) on each copy —
  the adjoint gradient at kappa != 0 (transposed solve) against the periodic one;
* dimensional scaling: every spacing times lambda, E and V over lambda^2, the projector
  couplings over lambda^5 (the h^3 of <p|psi> gives lambda^3) scale the whole discrete
  equation by 1 / lambda^2: T and R unchanged — every power of h in the FD weights, the
  self-energy coupling, the KB term and the velocities;
* a flat potential on an anisotropic grid (h_x, h_y, h_z all different, nx != ny):
  T = I, R = 0 — the electrodes' z-modes and the interior's z-couplings use the same h_z;
* unitarity of the flux-normalised scattering matrix S = [[r, t'], [t, r']] (left- and
  right-incident amplitudes scaled by sqrt(v_out / v_in)): S^H S = I, off-diagonal
  entries included, at kappa = 0 and at a Bloch vector kappa (both sides at the same
  kappa).  Current conservation T + R = 1 is its diagonal; the rest fixes the phases
  of the projected amplitudes (Eq. 6, Eq. 19) up to the diagonal phase conventions,
  which leave S unitary.

The potential is a wire of wells with a seeded random perturbation (no symmetry of
its own), with s/p Kleinman-Bylander projectors.
"""
import math

import numpy as np
import pytest

import iobm_synth as S
from oracle import transport


def junction(nx=8, ny=6, nz=18, h=0.6, nf=4, seed=5):
    jn = S.small_wire(nx=nx, ny=ny, nz=nz, h=h, natom=2, spacing=3.0, depth=0.6, width=0.9,
                      rs=1.4, kb_kinds=S.SP, nf=nf, seed=seed, kb_radius=1.4, kb_width=0.6)
    rng = np.random.default_rng(seed + 1)
    bump = 0.08 * rng.standard_normal(jn.V.shape)
    bump[:nf] = 0.0          # keep the end planes' potential as generated
    bump[-nf:] = 0.0
    return jn.copy_with(V=jn.V + bump)


def remap(jn, V, f, **grid):
    """Junction with potential V and every projector point (z, y, x) moved to the
    linear index f(z, y, x) of the new grid."""
    projs = []
    for p in jn.projectors:
        z, rem = np.divmod(p.idx.astype(np.int64), jn.nx * jn.ny)
        y, x = np.divmod(rem, jn.nx)
        idx = f(z, y, x)
        order = np.argsort(idx, kind="stable")
        projs.append(S.Projector(idx=idx[order].astype(np.int32), val=p.val[order],
                                 coupling=p.coupling, atom=p.atom))
    return jn.copy_with(V=np.ascontiguousarray(V), projectors=projs, **grid)


def supercell_x2(jn):
    """The cell doubled along x: V and every projector repeated in the second copy."""
    nx, ny = jn.nx, jn.ny
    projs = []
    for shift in (0, nx):   # two copies of every projector, one per original cell
        for p in jn.projectors:
            z, rem = np.divmod(p.idx.astype(np.int64), nx * ny)
            y, x = np.divmod(rem, nx)
            projs.append(S.Projector(idx=((z * ny + y) * 2 * nx + x + shift).astype(np.int32),
                                     val=p.val, coupling=p.coupling, atom=p.atom))
    return jn.copy_with(nx=2 * nx, V=np.concatenate([jn.V, jn.V], axis=2), projectors=projs)


def test_supercell_folds_two_bloch_vectors():
    jn = junction(nx=6, ny=6, nz=16, h=0.65)
    nx = jn.nx
    sup = supercell_x2(jn)
    for E in (jn.e_fermi - 0.05, jn.e_fermi + 0.03):
        g0 = transport.solve(jn, E)
        gpi = transport.solve(jn, E, kappa=(math.pi / (nx * jn.hx), 0.0))
        gs = transport.solve(sup, E)
        assert gs.n_open == g0.n_open + gpi.n_open
        assert g0.n_open > 0 and gpi.n_open > 0
        assert abs(gs.G - (g0.G + gpi.G)) < 1e-9, (gs.G, g0.G, gpi.G)


def test_supercell_gradient_folds_two_bloch_vectors():
    jn = junction(nx=6, ny=6, nz=16, h=0.65)
    nx = jn.nx
    E = jn.e_fermi - 0.05
    g0 = transport.grad_V(jn, E)
    gpi = transport.grad_V(jn, E, kappa=(math.pi / (nx * jn.hx), 0.0))
    gs = transport.grad_V(supercell_x2(jn), E)
    scale = np.max(np.abs(g0 + gpi))
    assert scale > 0
    assert np.max(np.abs(gs[:, :, :nx] - gs[:, :, nx:])) < 1e-10 * scale
    assert np.max(np.abs(2.0 * gs[:, :, :nx] - (g0 + gpi))) < 1e-10 * scale


def test_transposed_cell_same_conductance():
    jn = junction(nx=8, ny=6, nz=18)
    jn = jn.copy_with(hy=0.55)   # h_x != h_y as well as nx != ny
    tr = remap(jn, jn.V.transpose(0, 2, 1), lambda z, y, x: (z * jn.nx + x) * jn.ny + y,
               nx=jn.ny, ny=jn.nx, hx=jn.hy, hy=jn.hx)
    for E in (jn.e_fermi - 0.04, jn.e_fermi + 0.02):
        a, b = transport.solve(jn, E), transport.solve(tr, E)
        assert a.n_open == b.n_open and a.n_open > 1
        assert abs(a.G - b.G) < 1e-9
        # the channels pair up: the same set of per-channel transmissions
        assert np.allclose(np.sort(a.T.sum(axis=0)), np.sort(b.T.sum(axis=0)), atol=1e-9)


@pytest.mark.parametrize("sy,sx", [(1, 3), (5, 2)])
def test_lateral_translation_same_t_and_r(sy, sx):
    jn = junction(nx=8, ny=6, nz=18)
    sh = remap(jn, np.roll(jn.V, (sy, sx), axis=(1, 2)),
               lambda z, y, x: (z * jn.ny + (y + sy) % jn.ny) * jn.nx + (x + sx) % jn.nx)
    E = jn.e_fermi - 0.01
    a, b = transport.solve(jn, E), transport.solve(sh, E)
    assert np.array_equal(a.open_modes, b.open_modes)
    assert np.max(np.abs(a.T - b.T)) < 1e-9 and np.max(np.abs(a.R - b.R)) < 1e-9


@pytest.mark.parametrize("nf", [1, 4])
def test_mirror_image_swaps_the_electrodes(nf):
    jn = junction(nx=8, ny=6, nz=18, nf=nf)
    mi = remap(jn, jn.V[::-1], lambda z, y, x: ((jn.nz - 1 - z) * jn.ny + y) * jn.nx + x)
    E = jn.e_fermi + 0.01
    right = transport.solve(jn, E, side="R")
    left_of_mirror = transport.solve(mi, E, side="L")
    assert np.array_equal(right.open_modes, left_of_mirror.open_modes) and right.n_open > 1
    assert np.max(np.abs(right.T - left_of_mirror.T)) < 1e-9
    assert np.max(np.abs(right.R - left_of_mirror.R)) < 1e-9
    # the junction has no mirror symmetry of its own: the two sides reflect differently
    assert np.max(np.abs(transport.solve(jn, E, side="L").R - right.R)) > 1e-6


def scattering_matrix(jn, E, kappa=(0.0, 0.0)):
    L = transport.solve(jn, E, side="L", kappa=kappa)
    R = transport.solve(jn, E, side="R", kappa=kappa)
    f = np.sqrt(L.vel[:, None] / L.vel[None, :])
    return np.block([[L.r * f, R.t * f], [L.t * f, R.r * f]])


@pytest.mark.parametrize("nf", [1, 4])
@pytest.mark.parametrize("fk", [(0.0, 0.0), (0.37, -0.52)])
def test_scattering_matrix_unitary(nf, fk):
    jn = junction(nx=8, ny=6, nz=18, nf=nf)
    k = (fk[0] * math.pi / (jn.nx * jn.hx), fk[1] * math.pi / (jn.ny * jn.hy))
    for E in (jn.e_fermi - 0.03, jn.e_fermi + 0.01):
        S_ = scattering_matrix(jn, E, k)
        n2 = S_.shape[0]
        assert n2 >= 4
        assert np.max(np.abs(S_.conj().T @ S_ - np.eye(n2))) < 1e-10


@pytest.mark.parametrize("nf", [1, 4])
def test_dimensional_scaling(nf):
    jn = junction(nx=8, ny=6, nz=18, nf=nf).copy_with(hy=0.55, hz=0.5)
    lam = 1.37
    projs = [S.Projector(idx=p.idx, val=p.val, coupling=p.coupling / lam ** 5, atom=p.atom)
             for p in jn.projectors]
    sc = jn.copy_with(hx=jn.hx * lam, hy=jn.hy * lam, hz=jn.hz * lam, V=jn.V / lam ** 2,
                      projectors=projs)
    E = jn.e_fermi - 0.02
    a, b = transport.solve(jn, E), transport.solve(sc, E / lam ** 2)
    assert a.n_open == b.n_open and a.n_open > 1
    assert np.max(np.abs(a.T - b.T)) < 1e-10 and np.max(np.abs(a.R - b.R)) < 1e-10


@pytest.mark.parametrize("nf", [1, 4])
def test_flat_potential_anisotropic_grid(nf):
    jn = S.small_wire(nx=10, ny=9, nz=16, h=0.55, natom=1, depth=0.0, rs=1.4, nf=nf)
    jn = jn.copy_with(hy=0.62, hz=0.47, V=np.zeros_like(jn.V))
    sol = transport.solve(jn, jn.e_fermi)
    assert sol.n_open >= 3
    assert np.max(np.abs(sol.T - np.eye(sol.n_open))) < 1e-10
    assert np.max(np.abs(sol.R)) < 1e-10
