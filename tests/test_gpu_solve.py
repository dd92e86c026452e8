"""GPU solves against the oracle's exact (sparse-LU) solutions, through the C ABI.

Bar: conductance within 1e-6 G_0 of the oracle, every T and R entry within
1e-6, FP64 relative residual <= 1e-8 for every RHS, in both the plain FP64
solver and the mixed FP32/FP64 solver."""
import numpy as np
import pytest
import torch

import iobm_synth as S
from oracle import operator, transport

pytestmark = pytest.mark.gpu

G_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1009_5300_gb300 import build_library
    build_library()


def kb_junction(nf=4):
    return S.small_wire(nx=12, ny=12, nz=26, h=0.5, natom=2, spacing=3.4, depth=0.7, width=0.9,
                        rs=1.6, kb_kinds=S.SP, nf=nf, seed=77)


def compare(res, sol_or, tol=G_TOL):
    n = sol_or.n_open
    assert res.n_open[0] == n
    assert np.all(res.status == 0), res.status
    assert np.all(res.residual <= 1e-8), res.residual
    T = res.T[:, :n].T          # [out][in]
    R = res.R[:, :n].T
    assert np.max(np.abs(T - sol_or.T)) < tol
    assert np.max(np.abs(R - sol_or.R)) < tol
    assert abs(res.G[0] - sol_or.G) < tol


@pytest.fixture(scope="module")
def wire16_oracle():
    jn = S.wire16()
    return jn, transport.solve(jn, jn.energies[0])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_wire16(wire16_oracle, precision):
    from paper_1009_5300_gb300 import IOBMSolver
    jn, ref = wire16_oracle
    sol = IOBMSolver.from_junction(jn, precision=precision)
    res = sol.solve(jn.energies)
    compare(res, ref)
    # the solution itself against the oracle's
    psi = sol.solution(0).cpu().numpy()
    assert np.max(np.abs(psi - ref.psi[0])) < 1e-6 * np.max(np.abs(ref.psi[0]))
    sol.close()


@pytest.mark.parametrize("nf", [1, 4])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("precond", ["fourier", "fourier_explicit", "eq10"])
def test_multichannel_kb(nf, precision, precond):
    from paper_1009_5300_gb300 import IOBMSolver
    jn = kb_junction(nf)
    E = jn.e_fermi
    ref = transport.solve(jn, E)
    kw = {"use_precond": precond}
    if precond == "fourier_explicit":   # stencil + self-energy + projectors every iteration
        kw = {"use_precond": "fourier", "op_form": "explicit"}
    sol = IOBMSolver.from_junction(jn, precision=precision, **kw)
    res = sol.solve([E])
    assert ref.n_open >= 3
    compare(res, ref)
    # current conservation on the GPU result alone
    assert np.max(np.abs(res.T.sum(1) + res.R.sum(1) - 1.0)) < 1e-6
    sol.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_explicit_form_on_row_blocked_stencil(precision):
    # a 12 x 16 plane takes the row-blocked FP32 stencil (variant 0: fused p update,
    # operator and p^T A p over 16-row tiles) or the plane-ring kernel (variant 4) in
    # every explicit-form iteration: oracle T, R, G
    from paper_1009_5300_gb300 import IOBMSolver
    jn = S.small_wire(nx=12, ny=16, nz=30, h=0.5, natom=2, spacing=3.4, depth=0.7, width=0.9,
                      rs=1.6, kb_kinds=S.SP, nf=4, seed=78)
    E = jn.e_fermi
    ref = transport.solve(jn, E)
    for z, var in ((16, 0), (32, 0), (64, 0), (16, 4), (32, 4)):
        sol = IOBMSolver.from_junction(jn, precision=precision, op_form="explicit")
        sol.set_tiling(z, var)
        res = sol.solve([E])
        assert ref.n_open >= 3
        compare(res, ref)
        sol.close()


def test_eq10_fourier_form_solve():
    # the Fourier form of Eq. 10 drives the same Krylov iteration as the stencil form
    from paper_1009_5300_gb300 import IOBMSolver
    jn = kb_junction(4)
    E = jn.e_fermi
    ref = transport.solve(jn, E)
    its = []
    for precond in ("eq10", "eq10_fourier"):
        sol = IOBMSolver.from_junction(jn, precision="fp64", use_precond=precond, alpha=1.8)
        res = sol.solve([E])
        compare(res, ref)
        its.append(res.iterations)
        sol.close()
    # different rounding over ~200 Krylov steps moves the counts by a few per cent
    assert np.max(np.abs(its[0] - its[1])) <= 0.05 * np.max(its[0])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_implicit_operator_form(precision):
    # with the free-propagator preconditioner, q = A p formed as (r - V z) + beta q_old
    # - V_NL z drives the same Krylov iteration as the explicit operator: both reach
    # the oracle's solution, with iteration counts a rounding-level apart
    from paper_1009_5300_gb300 import IOBMSolver
    jn = kb_junction(4)
    Es = [jn.e_fermi - 0.02, jn.e_fermi]
    its, stage_ms = {}, {}
    for form in ("auto", "explicit"):
        sol = IOBMSolver.from_junction(jn, precision=precision, op_form=form)
        sol.profile("operator")
        res = sol.solve(Es)
        stage_ms[form] = sol.kernel_stats()
        sol.profile(False)
        assert res.converged, res.status
        assert np.all(res.residual <= 1e-8)
        for e, E in enumerate(Es):
            assert abs(res.G[e] - transport.conductance(jn, E)) < G_TOL
        its[form] = res.iterations.astype(float)
        sol.close()
    for form in its:
        assert stage_ms[form][1] > 0 and stage_ms[form][0] > 0
    assert its["auto"].mean() <= 1.2 * its["explicit"].mean() + 2


def test_replacement_steps_with_and_without_conditional_nodes(monkeypatch):
    # the FP64 residual replacements captured as IF nodes (default) and as plain masked
    # launches (IOBM_GRAPH_CONDITIONALS=0, read when a handle is created) run the same
    # kernels on the same RHS: bit-identical results
    from paper_1009_5300_gb300 import IOBMSolver
    jn = kb_junction(4)
    Es = [jn.e_fermi - 0.02, jn.e_fermi]
    out = []
    for flag in (None, "0"):
        if flag is None:
            monkeypatch.delenv("IOBM_GRAPH_CONDITIONALS", raising=False)
        else:
            monkeypatch.setenv("IOBM_GRAPH_CONDITIONALS", flag)
        sol = IOBMSolver.from_junction(jn, precision="mixed")
        res = sol.solve(Es)
        assert res.converged
        out.append(res)
        sol.close()
    assert np.array_equal(out[0].T, out[1].T)
    assert np.array_equal(out[0].R, out[1].R)
    assert np.array_equal(out[0].iterations, out[1].iterations)
    assert np.array_equal(out[0].replacements, out[1].replacements)


def test_profile_stages():
    # every timed stage of the fused Fourier preconditioner reports launches
    from paper_1009_5300_gb300 import IOBMSolver
    jn = kb_junction(4)
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    for stage in ("operator", "update_fft", "zsweep", "ifft"):
        sol.profile(stage)
        sol.solve([jn.e_fermi])
        ms, n = sol.kernel_stats()
        assert n > 0 and ms > 0, stage
    sol.profile(False)
    sol.close()


def test_precision_escalation():
    # with a tiny FP32 iteration limit every RHS stops unconverged in the mixed phase
    # and is finished by FP64 COCG from its FP64 iterate: same exact solution
    from paper_1009_5300_gb300 import IOBMSolver, solve_batch
    jn = kb_junction(4)
    E = jn.e_fermi
    ref = transport.solve(jn, E)
    sol = IOBMSolver.from_junction(jn, precision="mixed", max_iter_mixed=4)
    res = sol.solve([E])
    compare(res, ref)
    assert np.all(res.iterations > 4)
    sol.close()
    # the batched path escalates the same way
    sols = [IOBMSolver.from_junction(jn, precision="mixed", max_iter_mixed=4) for _ in range(2)]
    out = solve_batch(sols, [[E], [E - 0.02]])
    compare(out[0], ref)
    assert abs(out[1].G[0] - transport.conductance(jn, E - 0.02)) < G_TOL
    for s in sols:
        s.close()


def test_eigenchannels():
    # eigenvalues of T^dagger T from the library's FP64 amplitudes against the oracle's
    from paper_1009_5300_gb300 import IOBMSolver
    from paper_1009_5300_gb300._lib import IOBMError
    jn = kb_junction(4)
    E = jn.e_fermi
    ref = transport.solve(jn, E)
    tau_ref = transport.eigenchannels(ref)
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    res = sol.solve([E])
    tau = sol.eigenchannels(0)
    assert len(tau) == ref.n_open
    assert np.max(np.abs(tau - tau_ref)) < 1e-6
    assert abs(tau.sum() - res.G[0]) < 1e-9
    # a solve over a channel subset cannot give the transmission matrix
    sol.solve([E], channels=[0])
    with pytest.raises(IOBMError):
        sol.eigenchannels(0)
    sol.close()
    flat = S.small_wire(nx=12, ny=10, nz=20, h=0.6, natom=1, depth=0.0, rs=1.5, nf=4)
    flat = flat.copy_with(V=np.zeros_like(flat.V))
    sf = IOBMSolver.from_junction(flat, precision="mixed")
    sf.solve([flat.e_fermi])
    assert np.max(np.abs(sf.eigenchannels(0) - 1.0)) < 1e-6
    sf.close()


def test_right_incidence_and_reciprocity():
    from paper_1009_5300_gb300 import IOBMSolver
    jn = kb_junction(4)
    E = jn.e_fermi - 0.02
    refR = transport.solve(jn, E, side="R")
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    resR = sol.solve([E], side=1)
    compare(resR, refR)
    resL = sol.solve([E], side=0)
    assert abs(resL.G[0] - resR.G[0]) < 2 * G_TOL
    sol.close()


def test_flat_potential_integer_conductance():
    from paper_1009_5300_gb300 import IOBMSolver
    jn = S.small_wire(nx=12, ny=10, nz=20, h=0.6, natom=1, depth=0.0, rs=1.5, nf=4)
    jn = jn.copy_with(V=np.zeros_like(jn.V))
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    res = sol.solve([jn.e_fermi])
    n = res.n_open[0]
    assert n >= 3
    assert abs(res.G[0] - n) < G_TOL
    assert np.max(np.abs(res.T[:, :n] - np.eye(n))) < G_TOL
    sol.close()


def test_several_energies_and_batch_independence():
    from paper_1009_5300_gb300 import IOBMSolver
    jn = kb_junction(4)
    Es = [jn.e_fermi - 0.05, jn.e_fermi, jn.e_fermi + 0.03]
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    res = sol.solve(Es)
    for e, E in enumerate(Es):
        ref = transport.solve(jn, E)
        assert abs(res.G[e] - ref.G) < G_TOL
    # the same channel pair solved alone gives bit-identical results
    k = int(np.nonzero(res.energy_index == 1)[0][1])
    single = sol.solve([Es[1]], channels=[int(res.channel[k])])
    assert np.array_equal(single.T[0], res.T[k][: single.T.shape[1]])
    assert single.iterations[0] == res.iterations[k]
    sol.close()


def test_gradient_matches_oracle_and_fd():
    from paper_1009_5300_gb300 import IOBMSolver
    jn = S.small_wire(nx=8, ny=8, nz=20, h=0.6, natom=2, spacing=3.0, depth=0.6, width=0.9,
                      rs=1.4, kb_kinds=S.SP, nf=4, seed=5)
    E = jn.e_fermi
    ref = transport.grad_V(jn, E)
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    g, G = sol.grad_V(E)
    g = g.cpu().numpy()
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(g - ref)) < 1e-5 * scale
    assert abs(G - transport.conductance(jn, E)) < G_TOL
    sol.close()


def test_autograd_function():
    from paper_1009_5300_gb300 import IOBMSolver, conductance
    jn = S.small_wire(nx=8, ny=8, nz=20, h=0.6, natom=2, spacing=3.0, depth=0.6, width=0.9,
                      rs=1.4, nf=4, seed=9)
    E = jn.e_fermi
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    V = torch.tensor(jn.V, device="cuda", requires_grad=True)
    G = conductance(V, sol, E)
    G.backward()
    ref = transport.grad_V(jn, E)
    assert abs(G.item() - transport.conductance(jn, E)) < G_TOL
    assert np.max(np.abs(V.grad.cpu().numpy() - ref)) < 1e-5 * np.max(np.abs(ref))
    sol.close()
