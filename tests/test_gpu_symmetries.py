"""The oracle's symmetry pins reproduced by the CUDA path (mixed precision, through the
C ABI): transformed junctions solved on the GPU give the transformed results, and each
side agrees with the FP64 oracle to the 1e-6 G_0 bar.

* x <-> y transposition of a non-square cell with h_x != h_y: same G;
* lateral translation by whole grid steps: T and R unchanged entry by entry;
* the mirror image z -> -z: incidence from the left of the mirror = from the right of
  the original;
* the lateral supercell: G_super(kappa = 0) = G(0) + G(pi / L_x) of the original cell,
  the latter through the library's Bloch-vector solve;
* on large planes, GPU against GPU (no oracle at these sizes): a translation of a
  128 x 128 cell (on-chip CTA-pair transforms) and the transposition of a 128 x 64 cell
  (two-pass global-memory transforms).
"""
import math

import numpy as np
import pytest

import test_oracle_symmetries as TS
from oracle import transport

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1009_5300_gb300 import build_library
    build_library()


def gpu_solve(jn, E, side=0, kappa=None):
    from paper_1009_5300_gb300 import IOBMSolver
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    if kappa is not None:
        sol.set_bloch(kappa)
    res = sol.solve(list(E), side=side)
    sol.close()
    assert res.converged, res.status
    assert np.all(res.residual <= 1e-8)
    return res


def test_transposed_cell_same_conductance_on_gpu():
    jn = TS.junction(nx=8, ny=6, nz=18).copy_with(hy=0.55)
    tr = TS.remap(jn, jn.V.transpose(0, 2, 1), lambda z, y, x: (z * jn.nx + x) * jn.ny + y,
                  nx=jn.ny, ny=jn.nx, hx=jn.hy, hy=jn.hx)
    E = [jn.e_fermi - 0.04, jn.e_fermi + 0.02]
    a, b = gpu_solve(jn, E), gpu_solve(tr, E)
    for e, En in enumerate(E):
        ref = transport.solve(jn, En)
        assert a.n_open[e] == b.n_open[e] == ref.n_open
        assert abs(a.G[e] - ref.G) < TOL and abs(b.G[e] - ref.G) < TOL
        assert abs(a.G[e] - b.G[e]) < TOL


def test_lateral_translation_same_t_and_r_on_gpu():
    jn = TS.junction(nx=8, ny=6, nz=18)
    sy, sx = 1, 3
    sh = TS.remap(jn, np.roll(jn.V, (sy, sx), axis=(1, 2)),
                  lambda z, y, x: (z * jn.ny + (y + sy) % jn.ny) * jn.nx + (x + sx) % jn.nx)
    E = [jn.e_fermi - 0.01]
    a, b = gpu_solve(jn, E), gpu_solve(sh, E)
    assert np.array_equal(a.channel, b.channel)
    assert np.max(np.abs(a.T - b.T)) < TOL and np.max(np.abs(a.R - b.R)) < TOL
    ref = transport.solve(jn, E[0])
    n = ref.n_open
    for k in range(a.nrhs):
        assert np.max(np.abs(a.T[k, :n] - ref.T[:, int(a.channel[k])])) < TOL


@pytest.mark.parametrize("nf", [1, 4])
def test_mirror_image_swaps_the_electrodes_on_gpu(nf):
    jn = TS.junction(nx=8, ny=6, nz=18, nf=nf)
    mi = TS.remap(jn, jn.V[::-1], lambda z, y, x: ((jn.nz - 1 - z) * jn.ny + y) * jn.nx + x)
    E = [jn.e_fermi + 0.01]
    right = gpu_solve(jn, E, side=1)
    left_of_mirror = gpu_solve(mi, E, side=0)
    assert np.array_equal(right.channel, left_of_mirror.channel)
    assert np.max(np.abs(right.T - left_of_mirror.T)) < TOL
    assert np.max(np.abs(right.R - left_of_mirror.R)) < TOL
    assert abs(right.G[0] - transport.solve(jn, E[0], side="R").G) < TOL


def test_supercell_folds_two_bloch_vectors_on_gpu():
    jn = TS.junction(nx=6, ny=6, nz=16, h=0.65)
    nx, ny = jn.nx, jn.ny
    projs = []
    for shift in (0, nx):
        for p in jn.projectors:
            z, rem = np.divmod(p.idx.astype(np.int64), nx * ny)
            y, x = np.divmod(rem, nx)
            projs.append(TS.S.Projector(idx=((z * ny + y) * 2 * nx + x + shift).astype(np.int32),
                                        val=p.val, coupling=p.coupling, atom=p.atom))
    sup = jn.copy_with(nx=2 * nx, V=np.concatenate([jn.V, jn.V], axis=2), projectors=projs)
    E = [jn.e_fermi - 0.05]
    g0 = gpu_solve(jn, E)
    gpi = gpu_solve(jn, E, kappa=(math.pi / (nx * jn.hx), 0.0))   # slots: +kappa, -kappa
    gs = gpu_solve(sup, E)
    assert gs.n_open[0] == g0.n_open[0] + gpi.n_open[0]
    assert abs(gpi.G[0] - gpi.G[1]) < TOL        # pi / L_x and -pi / L_x: the same waves
    assert abs(gs.G[0] - (g0.G[0] + gpi.G[0])) < 2 * TOL
    assert abs(gs.G[0] - transport.solve(sup, E[0]).G) < TOL


def large_junction(nx, ny):
    import iobm_synth as S
    return S.small_wire(nx=nx, ny=ny, nz=20, h=0.3, natom=1, depth=0.4, width=1.0, rs=6.0,
                        kb_kinds=S.SP, nf=4, seed=9, kb_radius=1.4, kb_width=0.6)


def test_large_plane_translation_on_gpu():
    # 128 x 128 planes: the self-energy and the free propagator transform on chip in CTA
    # pairs; a lateral translation must leave T and R unchanged entry by entry
    jn = large_junction(128, 128)
    sy, sx = 37, 91
    sh = TS.remap(jn, np.roll(jn.V, (sy, sx), axis=(1, 2)),
                  lambda z, y, x: (z * jn.ny + (y + sy) % jn.ny) * jn.nx + (x + sx) % jn.nx)
    E = [jn.e_fermi]
    a, b = gpu_solve(jn, E), gpu_solve(sh, E)
    assert a.nrhs > 1 and np.array_equal(a.channel, b.channel)
    assert np.max(np.abs(a.T - b.T)) < TOL and np.max(np.abs(a.R - b.R)) < TOL


def test_large_plane_transposition_on_gpu():
    # 128 x 64 planes (above 4096 points: the two-pass global-memory transforms) and
    # their 64 x 128 transpose: the same conductance
    jn = large_junction(128, 64)
    tr = TS.remap(jn, jn.V.transpose(0, 2, 1), lambda z, y, x: (z * jn.nx + x) * jn.ny + y,
                  nx=jn.ny, ny=jn.nx, hx=jn.hy, hy=jn.hx)
    E = [jn.e_fermi]
    a, b = gpu_solve(jn, E), gpu_solve(tr, E)
    assert a.n_open[0] == b.n_open[0] > 1
    assert abs(a.G[0] - b.G[0]) < TOL
