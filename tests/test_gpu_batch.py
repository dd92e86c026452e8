"""Batched solves of several junctions of uneven size (one graph launch with a
device-side WHILE loop per junction), through the C ABI.

Bars: a junction solved in a batch gives bit-identical T, R and iteration counts
to the same junction solved alone (same tiling); batched conductances match the
oracle's exact solutions within 1e-6 G_0; with autotuned tiling (a different
order of the partial sums) within 1e-6 G_0 of the untuned results; on a sample of
the full-size uneven-batch generator (lateral 24-64, N_z 96-256) every RHS
converges, T + R = 1 per incident channel, and a sampled wave of each junction has
an FP64 residual <= 1e-8 under the oracle's matrix-free operator."""
import numpy as np
import pytest

import iobm_synth as S
from oracle import modes, operator, transport

pytestmark = pytest.mark.gpu
G_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1009_5300_gb300 import build_library
    build_library()


def small_junctions():
    a = S.small_wire(nx=12, ny=12, nz=26, h=0.5, natom=2, spacing=3.4, depth=0.7, width=0.9,
                     rs=1.6, kb_kinds=S.SP, nf=4, seed=77)
    b = S.small_wire(nx=16, ny=16, nz=30, h=0.5, natom=2, spacing=3.0, depth=0.6, width=1.0,
                     rs=1.8, nf=4, seed=5)
    c = S.small_wire(nx=10, ny=10, nz=20, h=0.6, natom=1, depth=0.5, width=0.9, rs=1.5, nf=1,
                     seed=9)
    return [a, b, c]


def energies_of(jn):
    return [jn.e_fermi - 0.02, jn.e_fermi + 0.01]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_matches_individual_bitwise(precision):
    from paper_1009_5300_gb300 import IOBMSolver, solve_batch
    jns = small_junctions()
    alone = []
    for jn in jns:
        s = IOBMSolver.from_junction(jn, precision=precision)
        alone.append(s.solve(energies_of(jn)))
        s.close()
    sols = [IOBMSolver.from_junction(jn, precision=precision) for jn in jns]
    batch = solve_batch(sols, [energies_of(jn) for jn in jns])
    for ra, rb in zip(alone, batch):
        assert rb.converged, rb.status
        assert np.array_equal(ra.T, rb.T)
        assert np.array_equal(ra.R, rb.R)
        assert np.array_equal(ra.iterations, rb.iterations)
        assert np.array_equal(ra.G, rb.G)
    for s in sols:
        s.close()


def test_batch_against_oracle_and_autotune():
    from paper_1009_5300_gb300 import IOBMSolver, solve_batch
    jns = small_junctions()
    sols = [IOBMSolver.from_junction(jn, precision="mixed") for jn in jns]
    batch = solve_batch(sols, [energies_of(jn) for jn in jns])
    for jn, res in zip(jns, batch):
        for e, E in enumerate(energies_of(jn)):
            assert abs(res.G[e] - transport.conductance(jn, E)) < G_TOL
    tuned = [IOBMSolver.from_junction(jn, precision="mixed") for jn in jns]
    batch2 = solve_batch(tuned, [energies_of(jn) for jn in jns], autotune=True)
    for r1, r2 in zip(batch, batch2):
        assert r2.converged
        assert np.max(np.abs(r1.G - r2.G)) < G_TOL
    for s in sols + tuned:
        s.close()


def test_tiling_choices_agree():
    # every (z-chunk, kernel) choice the autotuner can make gives the same solution
    from paper_1009_5300_gb300 import IOBMSolver
    jn = small_junctions()[1]
    ref = None
    for zc, var in [(32, 0), (16, 0), (64, 0), (16, 1), (32, 1)]:
        s = IOBMSolver.from_junction(jn, precision="mixed")
        s.set_tiling(zc, var)
        r = s.solve(energies_of(jn))
        assert r.converged
        if ref is None:
            ref = r
        else:
            assert np.max(np.abs(r.G - ref.G)) < G_TOL
        s.close()


def test_uneven_full_size_sample():
    from paper_1009_5300_gb300 import IOBMSolver, solve_batch
    ids = [0, 1, 2, 3]
    jns = [S.batch_junction(j) for j in ids]
    Es = [jn.energies[[3, 12]] for jn in jns]
    sols = [IOBMSolver.from_junction(jn, precision="mixed") for jn in jns]
    results = solve_batch(sols, Es, autotune=True)
    for jn, E, sol, res in zip(jns, Es, sols, results):
        assert res.converged, (jn.name, res.status)
        assert np.all(res.residual <= 1e-8)
        for i in range(res.nrhs):
            n = res.n_open[res.energy_index[i]]
            assert abs(res.T[i, :n].sum() + res.R[i, :n].sum() - 1.0) < 1e-6
        k = res.nrhs // 2
        e = int(res.energy_index[k])
        c = int(res.channel[k])
        md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, jn.nf, float(E[e]))
        m = md.open_modes[c]
        psi = sol.solution(k).cpu().numpy()
        b = transport.source_vector(jn, md, m, "L", matrix_free=True)
        r = b - operator.apply_A(jn, float(E[e]), md, psi)
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
        sol.close()


def test_batch_rejects_duplicate_handles():
    from paper_1009_5300_gb300 import IOBMSolver, solve_batch
    from paper_1009_5300_gb300._lib import IOBMError
    jn = small_junctions()[2]
    s = IOBMSolver.from_junction(jn, precision="mixed")
    with pytest.raises(IOBMError):
        solve_batch([s, s], [energies_of(jn), energies_of(jn)])
    s.close()


def test_create_batch_abi():
    # iobm_create_batch makes independent handles; an invalid junction leaves none behind
    import ctypes as C
    from paper_1009_5300_gb300 import _lib
    lib = _lib.load()
    jns = small_junctions()[1:]
    n = len(jns)
    grids = (_lib.Grid * n)(*[_lib.Grid(j.nx, j.ny, j.nz, j.hx, j.hy, j.hz, j.nf) for j in jns])
    Vs = [np.ascontiguousarray(j.V, np.float64) for j in jns]
    vptr = (C.c_void_p * n)(*[v.ctypes.data for v in Vs])
    rs = (C.c_double * n)(*[j.rs for j in jns])
    opts = _lib.Options()
    lib.iobm_default_options(C.byref(opts))
    out = (C.c_void_p * n)()
    assert lib.iobm_create_batch(n, grids, vptr, None, rs, C.byref(opts), None, out) == 0
    for j, h in zip(jns, out):
        assert h
        k = C.c_int(0)
        assert lib.iobm_open_channels(h, float(j.e_fermi), C.byref(k), 0, None, None) == 0
        assert k.value >= 1
        lib.iobm_destroy(h)
    grids[1].nz = 2            # too few planes for N_f: rejected before any allocation
    out2 = (C.c_void_p * n)()
    assert lib.iobm_create_batch(n, grids, vptr, None, rs, C.byref(opts), None, out2) == _lib.IOBM_E_ARG
    assert not out2[0] and not out2[1]
