"""Lateral planes above 4096 points (two-pass global-memory FFTs for the
self-energy and the free-propagator preconditioner), through the C ABI.

The oracle's dense Eq. 8 blocks and sparse LU do not fit these sizes, so parity
uses what holds at any size: the preconditioner inverts the oracle's
potential-free operator (FP64 to 1e-10), every returned wave has an FP64
residual <= 1e-8 under the oracle's matrix-free operator (its Eq. 19 sums by FFT,
pinned to the explicit sums on small planes), T + R = 1 per incident channel,
and the mixed solver matches the plain FP64 solver within 1e-6 G_0.  The last
case is the 128 x 128 x 256 large cross-section workload at E_F (a sample of its
109 channels)."""
import numpy as np
import pytest
import torch

import iobm_synth as S
from oracle import modes, operator, transport

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1009_5300_gb300 import build_library
    build_library()


@pytest.mark.parametrize("nx,ny,nz,nf", [(72, 72, 20, 4), (96, 48, 16, 2)])
def test_large_plane_preconditioner_inverts_free_operator(nx, ny, nz, nf):
    from paper_1009_5300_gb300 import IOBMSolver
    jn = S.small_wire(nx=nx, ny=ny, nz=nz, h=0.45, natom=1, depth=0.7, width=1.0, rs=2.0,
                      kb_kinds=S.SP, nf=nf, seed=3)
    E = jn.e_fermi + 0.007
    md = modes.mode_data(nx, ny, jn.hx, jn.hy, jn.hz, nf, E)
    sol = IOBMSolver.from_junction(jn, precision="fp64", use_precond="fourier")
    x = np.stack([S.random_field((nz, ny, nx), 41 + i) for i in range(2)])
    xd = torch.from_numpy(x).cuda()
    free = jn.copy_with(V=np.zeros_like(jn.V), projectors=[])
    y = sol.apply_precond(xd, E).cpu().numpy()
    back = np.stack([operator.apply_A(free, E, md, y[i]) for i in range(2)])
    assert np.max(np.abs(back - x)) < 1e-10 * np.max(np.abs(x))
    y32 = sol.apply_precond(xd.to(torch.complex64), E).cpu().numpy()
    back32 = np.stack([operator.apply_A(free, E, md, y32[i]) for i in range(2)])
    assert np.max(np.abs(back32 - x)) < 1e-3 * np.max(np.abs(x))
    sol.close()


@pytest.mark.parametrize("nf", [4, 2])
def test_cluster_plane_transform_matches_oracle(nf):
    # 128 x 128 FP32 planes: forward and inverse transforms on chip by CTA pairs (the
    # column passes read the peer's rows through distributed shared memory); against the
    # oracle's per-mode banded free propagator, with the FP64 two-pass path beside it
    from oracle import iterative
    from paper_1009_5300_gb300 import IOBMSolver
    n, nz = 128, 11
    jn = S.small_wire(nx=n, ny=n, nz=nz, h=0.3, natom=1, depth=0.7, width=1.0, rs=2.0, nf=nf,
                      seed=13)
    E = jn.e_fermi + 0.004
    md = modes.mode_data(n, n, jn.hx, jn.hy, jn.hz, nf, E)
    x = np.stack([S.random_field((nz, n, n), 71 + i) for i in range(3)])
    ref = np.stack([iterative.free_propagator_modes(jn, E, md, xi) for xi in x])
    scale = np.max(np.abs(ref))
    sol = IOBMSolver.from_junction(jn, precision="fp64", use_precond="fourier")
    xd = torch.from_numpy(x).cuda()
    y64 = sol.apply_precond(xd, E).cpu().numpy()
    assert np.max(np.abs(y64 - ref)) < 1e-11 * scale
    y32 = sol.apply_precond(xd.to(torch.complex64), E).cpu().numpy()
    assert np.max(np.abs(y32 - ref)) < 1e-4 * scale
    sol.close()


def check_solution(jn, E, sol, res, k):
    e = int(res.energy_index[k])
    c = int(res.channel[k])
    md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, jn.nf, float(E[e]))
    m = md.open_modes[c]
    psi = sol.solution(k).cpu().numpy()
    b = transport.source_vector(jn, md, m, "L", matrix_free=True)
    r = b - operator.apply_A(jn, float(E[e]), md, psi)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8


def test_large_plane_solve():
    from paper_1009_5300_gb300 import IOBMSolver
    jn = S.small_wire(nx=72, ny=72, nz=30, h=0.5, natom=2, spacing=4.0, depth=0.6, width=1.0,
                      rs=1.6, kb_kinds=S.SP, nf=4, seed=8)
    E = np.array([jn.e_fermi])
    chans = [0, 1, 2, 5]
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    res = sol.solve(E, channels=chans)
    assert res.converged, res.status
    assert np.all(res.residual <= 1e-8)
    n = res.n_open[0]
    assert np.max(np.abs(res.T[:, :n].sum(1) + res.R[:, :n].sum(1) - 1.0)) < 1e-6
    check_solution(jn, E, sol, res, 1)
    s64 = IOBMSolver.from_junction(jn, precision="fp64")
    r64 = s64.solve(E, channels=chans)
    assert r64.converged
    assert abs(r64.G[0] - res.G[0]) < 1e-6
    s64.close()
    sol.close()


def test_large_cross_section_workload_sample():
    # the 128 x 128 x 256 wire (deep wells, s/p/d projectors, r_s = 2) at E_F
    from paper_1009_5300_gb300 import IOBMSolver
    jn = S.wire128()
    E = np.array([jn.e_fermi])
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    res = sol.solve(E, channels=[0, 54, 108])
    assert res.n_open[0] == 109
    assert res.converged, res.status
    assert np.all(res.residual <= 1e-8)
    n = res.n_open[0]
    assert np.max(np.abs(res.T[:, :n].sum(1) + res.R[:, :n].sum(1) - 1.0)) < 1e-6
    check_solution(jn, E, sol, res, 0)
    sol.close()
