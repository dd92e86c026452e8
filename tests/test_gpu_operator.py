"""GPU parity of the operator kernels against the oracle (called through the C ABI).

(E - H_T - H~) x: the z-marching FD stencil + local potential, the KB term and
the self-energy applied with lateral FFTs in clusters of N_f CTAs; P x: the
preconditioner of Eq. 10.  Sizes span several lateral tiles and z-chunks with
ragged tails."""
import numpy as np
import pytest
import torch

import iobm_synth as S
from oracle import modes, operator

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1009_5300_gb300 import build_library
    build_library()


def make(nx, ny, nz, nf, kb, h=0.45, seed=3):
    natom = 2 if nz >= 30 else 1
    return S.small_wire(nx=nx, ny=ny, nz=nz, h=h, natom=natom, spacing=3.0, depth=0.7, width=1.0,
                        rs=2.0, kb_kinds=S.SP if kb else None, nf=nf, seed=seed)


CASES = [
    (40, 12, 70, 4, True),     # 2 x 2 tiles with ragged x/y tails, 3 z-chunks (ragged)
    (6, 5, 9, 1, False),       # N_f = 1, one partial tile, odd lateral sizes
    (48, 48, 40, 4, True),     # the 48 x 48 lateral plane of the wire workload
    (25, 27, 36, 2, False),    # radix-5 and radix-3 FFTs, N_f = 2
    (64, 64, 12, 3, False),    # largest supported plane
    (80, 40, 20, 4, False),    # wider than the full-row stencil tiles: 2-D tiled kernel
    (3, 20, 12, 1, False),     # narrower than the full-row stencil tiles: 2-D tiled kernel
    (16, 16, 14, 1, True),     # compile-time-FFT self-energy with N_f = 1 (cluster of one CTA)
    (32, 32, 18, 2, False),    # compile-time-FFT self-energy, radix 4 and 2 passes, N_f = 2
    (72, 72, 14, 4, True),     # planes above 4096 points: two-pass global-memory FFTs
    (96, 48, 16, 2, True),     # a large non-square plane, 2-D tiled stencil (nx > 64)
    (24, 32, 37, 4, True),     # row-blocked FP32 kernel: 2 tiles of 16 rows, ragged z-chunk
    (64, 16, 29, 1, False),    # row-blocked kernel, N_f = 1, widest rows
    (12, 48, 21, 4, False),    # row-blocked kernel, narrowest rows, 3 tiles in y
]


@pytest.mark.parametrize("nx,ny,nz,nf,kb", CASES)
def test_apply_matches_oracle(nx, ny, nz, nf, kb):
    from paper_1009_5300_gb300 import IOBMSolver
    jn = make(nx, ny, nz, nf, kb)
    E = jn.e_fermi + 0.013
    sol = IOBMSolver.from_junction(jn, precision="fp64")
    md = modes.mode_data(nx, ny, jn.hx, jn.hy, jn.hz, nf, E)
    nrhs = 3
    x = np.stack([S.random_field((nz, ny, nx), 100 + i) for i in range(nrhs)])
    ref = np.stack([operator.apply_A(jn, E, md, x[i]) for i in range(nrhs)])
    xd = torch.from_numpy(x).cuda()
    y64 = sol.apply(E, xd).cpu().numpy()
    err64 = np.max(np.abs(y64 - ref)) / np.max(np.abs(ref))
    assert err64 < 1e-12, err64
    y32 = sol.apply(E, xd.to(torch.complex64)).cpu().numpy()
    err32 = np.max(np.abs(y32 - ref)) / np.max(np.abs(ref))
    assert err32 < 2e-5, err32
    # double-float stencil on FP64 data (the mixed solver's FP64 residual)
    ydf = sol.apply(E, xd, double_float=True).cpu().numpy()
    errdf = np.max(np.abs(ydf - ref)) / np.max(np.abs(ref))
    assert errdf < 1e-12, errdf
    sol.close()


@pytest.mark.parametrize("scale", [1e-6, 1.0, 1e6])
def test_double_float_apply_on_smooth_fields(scale):
    # smooth fields make the FD taps cancel against the diagonal; the double-float
    # arithmetic must still match FP64 to 1e-12 of the largest term, at any magnitude
    from paper_1009_5300_gb300 import IOBMSolver
    jn = make(48, 48, 40, 4, True)
    E = jn.e_fermi + 0.013
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    z, y, x = np.meshgrid(np.arange(jn.nz), np.arange(jn.ny), np.arange(jn.nx), indexing="ij")
    f = scale * (np.cos(2 * np.pi * x / jn.nx) * np.exp(1j * 2 * np.pi * y / jn.ny)
                 * np.sin(0.05 * z + 0.3) + 0.5)
    xd = torch.from_numpy(np.ascontiguousarray(f[None].astype(np.complex128))).cuda()
    y64 = sol.apply(E, xd).cpu().numpy()
    ydf = sol.apply(E, xd, double_float=True).cpu().numpy()
    big = scale * 0.5 * 3 * 1.4 / jn.hx ** 2          # size of the diagonal term
    assert np.max(np.abs(ydf - y64)) < 1e-12 * big
    sol.close()


@pytest.mark.parametrize("nx,ny,nz,nf,kb", CASES[:3] + CASES[-3:])
def test_precond_matches_oracle(nx, ny, nz, nf, kb):
    from paper_1009_5300_gb300 import IOBMSolver
    jn = make(nx, ny, nz, nf, kb)
    for alpha in (1.8, 3.0):
        sol = IOBMSolver.from_junction(jn, precision="fp64", alpha=alpha, use_precond="eq10")
        x = np.stack([S.random_field((nz, ny, nx), 7 + i) for i in range(2)])
        ref = np.stack([operator.apply_P(jn, alpha, x[i]) for i in range(2)])
        y = sol.apply_precond(torch.from_numpy(x).cuda()).cpu().numpy()
        assert np.max(np.abs(y - ref)) < 1e-13 * np.max(np.abs(ref))
        y32 = sol.apply_precond(torch.from_numpy(x).cuda().to(torch.complex64)).cpu().numpy()
        assert np.max(np.abs(y32 - ref)) < 1e-6 * np.max(np.abs(ref))
        sol.close()


@pytest.mark.parametrize("nx,ny,nz,nf,kb", [(20, 12, 30, 4, True), (16, 16, 24, 4, False),
                                             (25, 27, 16, 2, False), CASES[1]])
def test_eq10_fourier_form_matches_stencil(nx, ny, nz, nf, kb):
    # Eq. 10 applied through the lateral FFT (per-mode tridiagonal z-multiply) is the
    # operator of the real-space stencil form, to rounding; both against the oracle
    from paper_1009_5300_gb300 import IOBMSolver
    jn = make(nx, ny, nz, nf, kb)
    for alpha in (1.8, 3.0):
        st = IOBMSolver.from_junction(jn, precision="fp64", alpha=alpha, use_precond="eq10")
        ft = IOBMSolver.from_junction(jn, precision="fp64", alpha=alpha, use_precond="eq10_fourier")
        x = np.stack([S.random_field((nz, ny, nx), 11 + i) for i in range(2)])
        ref = np.stack([operator.apply_P(jn, alpha, x[i]) for i in range(2)])
        xd = torch.from_numpy(x).cuda()
        y_st = st.apply_precond(xd).cpu().numpy()
        y_ft = ft.apply_precond(xd).cpu().numpy()
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(y_ft - y_st)) < 1e-13 * scale
        assert np.max(np.abs(y_ft - ref)) < 1e-13 * scale
        y32 = ft.apply_precond(xd.to(torch.complex64)).cpu().numpy()
        assert np.max(np.abs(y32 - ref)) < 1e-6 * scale
        st.close()
        ft.close()


@pytest.mark.parametrize("nx,ny,nz,nf,kb", [(20, 12, 30, 4, True), CASES[1], (25, 27, 16, 2, False),
                                             (16, 16, 24, 4, True), (12, 12, 30, 1, False)])
def test_fourier_precond_matches_oracle(nx, ny, nz, nf, kb):
    # non-square and odd planes take the generic FFT, 16x16 and 12x12 the compile-time plans
    # (E - T - H~)^{-1} by lateral FFT + constant-factor z-sweeps against sparse LU
    from paper_1009_5300_gb300 import IOBMSolver
    jn = make(nx, ny, nz, nf, kb)
    E = jn.e_fermi + 0.007
    md = modes.mode_data(nx, ny, jn.hx, jn.hy, jn.hz, nf, E)
    sol = IOBMSolver.from_junction(jn, precision="fp64", use_precond="fourier")
    x = np.stack([S.random_field((nz, ny, nx), 31 + i) for i in range(2)])
    ref = operator.free_inverse(jn, E, md, x)
    y = sol.apply_precond(torch.from_numpy(x).cuda(), E).cpu().numpy()
    assert np.max(np.abs(y - ref)) < 1e-11 * np.max(np.abs(ref))
    y32 = sol.apply_precond(torch.from_numpy(x).cuda().to(torch.complex64), E).cpu().numpy()
    assert np.max(np.abs(y32 - ref)) < 1e-4 * np.max(np.abs(ref))
    sol.close()


@pytest.mark.parametrize("nx,ny,nz,nf,kb", [(24, 32, 37, 4, True), (64, 16, 29, 1, False),
                                             (12, 48, 21, 4, False), (48, 48, 40, 4, True),
                                             (16, 16, 12, 4, False)])
def test_ring_stencil_matches_oracle(nx, ny, nz, nf, kb):
    # variant 4: operand planes in a shared-memory ring (z-chunks of 16 and 32: ragged
    # last chunks, several tiles in y, the y-wrap split into up to three copies when the
    # tile with its halo is taller than the plane)
    from paper_1009_5300_gb300 import IOBMSolver
    jn = make(nx, ny, nz, nf, kb)
    E = jn.e_fermi + 0.013
    md = modes.mode_data(nx, ny, jn.hx, jn.hy, jn.hz, nf, E)
    x = np.stack([S.random_field((nz, ny, nx), 500 + i) for i in range(3)])
    ref = np.stack([operator.apply_A(jn, E, md, xi) for xi in x])
    scale = np.max(np.abs(ref))
    xd = torch.from_numpy(x).cuda().to(torch.complex64)
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    y0 = sol.apply(E, xd).cpu().numpy()
    for zc in (16, 32):
        sol.set_tiling(zc, 4)
        y4 = sol.apply(E, xd).cpu().numpy()
        assert np.max(np.abs(y4 - ref)) < 2e-5 * scale
        assert np.max(np.abs(y4 - y0)) < 2e-6 * scale
    sol.close()


@pytest.mark.parametrize("n,nz,nf", [(32, 14, 2), (48, 12, 4), (64, 10, 3)])
def test_two_factor_inverse_transform_matches_oracle(n, nz, nf):
    # square planes of 32, 48, 64 points take the two-factor inverse transform
    # (8 x 4, 12 x 4, 16 x 4); the oracle is its per-mode banded free propagator,
    # pinned against sparse LU on small grids
    from oracle import iterative
    from paper_1009_5300_gb300 import IOBMSolver
    jn = make(n, n, nz, nf, False)
    E = jn.e_fermi + 0.011
    md = modes.mode_data(n, n, jn.hx, jn.hy, jn.hz, nf, E)
    x = np.stack([S.random_field((nz, n, n), 61 + i) for i in range(2)])
    ref = np.stack([iterative.free_propagator_modes(jn, E, md, xi) for xi in x])
    scale = np.max(np.abs(ref))
    sol = IOBMSolver.from_junction(jn, precision="fp64", use_precond="fourier")
    y = sol.apply_precond(torch.from_numpy(x).cuda(), E).cpu().numpy()
    assert np.max(np.abs(y - ref)) < 1e-11 * scale
    y32 = sol.apply_precond(torch.from_numpy(x).cuda().to(torch.complex64), E).cpu().numpy()
    assert np.max(np.abs(y32 - ref)) < 1e-4 * scale
    sol.close()


def test_projector_on_end_planes_rejected():
    from paper_1009_5300_gb300 import IOBMSolver
    from paper_1009_5300_gb300._lib import IOBMError, IOBM_E_PROJ_BOUNDARY
    jn = make(12, 12, 30, 4, True)
    p = jn.projectors[0]
    bad = S.Projector(idx=np.array([5], np.int32), val=np.array([1.0]), coupling=0.1, atom=0)
    jn2 = jn.copy_with(projectors=[p, bad])
    with pytest.raises(IOBMError) as ei:
        IOBMSolver.from_junction(jn2)
    assert ei.value.code == IOBM_E_PROJ_BOUNDARY


def test_nonfinite_potential_rejected():
    from paper_1009_5300_gb300 import IOBMSolver
    from paper_1009_5300_gb300._lib import IOBMError, IOBM_E_ARG
    jn = make(8, 8, 12, 1, False)
    V = jn.V.copy()
    V[3, 2, 1] = np.nan
    with pytest.raises(IOBMError) as ei:
        IOBMSolver.from_junction(jn.copy_with(V=V))
    assert ei.value.code == IOBM_E_ARG
