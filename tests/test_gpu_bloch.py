"""GPU parity at a lateral Bloch vector kappa != 0 (Eq. 8: modes G_nu + kappa, the
wave picking up exp(i kappa L) across a lateral period), where A(kappa)^T = A(-kappa)
and the library runs preconditioned Bi-CG in the gauge phi = exp(-i kappa.r) psi,
the shadow sequence solving the -kappa problem.  Everything is compared with the
FP64 oracle at kappa (sparse LU, the Bloch-wrapped matrix-free operator, the
transposed adjoint), and the oracle's Bloch pins are reproduced on the GPU: flat
potential T = identity, T + R = 1 per incident channel, reciprocity
kappa <-> -kappa with reversed labels, the reciprocal-lattice shift."""
import math

import numpy as np
import pytest
import torch

import iobm_synth as S
from oracle import modes, operator, transport

pytestmark = pytest.mark.gpu

G_TOL = 1e-6


def kappa_of(jn, fx, fy):
    """kappa as fractions of the first Brillouin-zone half-width pi / L."""
    return (fx * math.pi / (jn.nx * jn.hx), fy * math.pi / (jn.ny * jn.hy))


def kb_junction(nf=4):
    return S.small_wire(nx=12, ny=12, nz=26, h=0.5, natom=2, spacing=3.4, depth=0.7, width=0.9,
                        rs=1.6, kb_kinds=S.SP, nf=nf, seed=77)


def gauge(jn, k, sign=1):
    """exp(i sign kappa.r) on the lateral plane, broadcast over [nz][ny][nx]."""
    x = np.arange(jn.nx) * jn.hx
    y = np.arange(jn.ny) * jn.hy
    return np.exp(1j * sign * (k[1] * y[:, None] + k[0] * x[None, :]))[None]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1009_5300_gb300 import build_library
    build_library()


@pytest.mark.parametrize("shape", [(12, 12, 26), (72, 8, 14)])
def test_operator_at_kappa_matches_oracle(shape):
    # rows kernel (nx <= 64) and the 2-D tile kernel (nx > 64), s/p projectors
    from paper_1009_5300_gb300 import IOBMSolver
    nx, ny, nz = shape
    jn = S.small_wire(nx=nx, ny=ny, nz=nz, h=0.45, natom=1, depth=0.6, width=0.9, rs=1.6,
                      kb_kinds=S.SP, kb_radius=1.3, kb_width=0.6, nf=4, seed=5)
    E = jn.e_fermi - 0.01
    k = kappa_of(jn, 0.37, -0.61)
    md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, 4, E, kappa=k)
    psi = np.stack([S.random_field((nz, ny, nx), 90 + i) for i in range(2)])
    ref = np.stack([operator.apply_A(jn, E, md, p) for p in psi])
    sol = IOBMSolver.from_junction(jn, precision="fp64")
    sol.set_bloch(k)
    phi = torch.from_numpy(psi * gauge(jn, k, -1)).cuda()
    y = sol.apply(E, phi).cpu().numpy() * gauge(jn, k, +1)
    assert np.max(np.abs(y - ref)) < 1e-12 * np.max(np.abs(ref))
    # the free propagator (E - T - H~)^{-1} at kappa
    z = sol.apply_precond(phi, E).cpu().numpy() * gauge(jn, k, +1)
    zref = operator.free_inverse(jn, E, md, psi)
    assert np.max(np.abs(z - zref)) < 1e-11 * np.max(np.abs(zref))
    sol.close()


def _compare(res, sol_ref, e_slot, tol=G_TOL):
    rows = np.nonzero(res.energy_index == e_slot)[0]
    n = sol_ref.n_open
    assert res.n_open[e_slot] == n and len(rows) == n
    assert abs(res.G[e_slot] - sol_ref.G) < tol, (res.G[e_slot], sol_ref.G)
    for k in rows:
        c = int(res.channel[k])
        assert np.max(np.abs(res.T[k, :n] - sol_ref.T[:, c])) < tol
        assert np.max(np.abs(res.R[k, :n] - sol_ref.R[:, c])) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_at_kappa_matches_oracle_both_signs(precision):
    from paper_1009_5300_gb300 import IOBMSolver
    jn = kb_junction()
    E = jn.e_fermi
    k = kappa_of(jn, 0.41, -0.27)
    ref_p = transport.solve(jn, E, kappa=k)
    ref_m = transport.solve(jn, E, kappa=(-k[0], -k[1]))
    sol = IOBMSolver.from_junction(jn, precision=precision)
    sol.set_bloch(k)
    res = sol.solve([E])
    assert res.converged, res.status
    assert np.all(res.residual <= 1e-8)
    print(f"{precision} at kappa: G {res.G[0]:.10f} (oracle {ref_p.G:.10f}), -kappa "
          f"{res.G[1]:.10f} ({ref_m.G:.10f}), iterations {res.iterations.tolist()}")
    _compare(res, ref_p, 0)
    _compare(res, ref_m, 1)
    # current conservation per incident channel, both signs
    for i in range(res.nrhs):
        n = res.n_open[res.energy_index[i]]
        assert abs(res.T[i, :n].sum() + res.R[i, :n].sum() - 1.0) < G_TOL
    # every returned wave (gauge undone) has oracle-operator residual <= 1e-8
    for i in range(res.nrhs):
        kk = k if res.energy_index[i] == 0 else (-k[0], -k[1])
        md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, 4, E, kappa=kk)
        m = md.open_modes[int(res.channel[i])]
        psi = sol.solution(i).cpu().numpy()
        b = transport.source_vector(jn, md, m, "L", matrix_free=True)
        r = b - operator.apply_A(jn, E, md, psi)
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
    sol.close()


@pytest.mark.parametrize("nf", [1, 4])
def test_flat_potential_at_kappa(nf):
    from paper_1009_5300_gb300 import IOBMSolver
    jn = S.small_wire(nx=12, ny=10, nz=14, h=0.6, natom=1, depth=0.0, rs=1.5, nf=nf)
    jn = jn.copy_with(V=np.zeros_like(jn.V))
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    sol.set_bloch(kappa_of(jn, 0.45, -0.7))
    res = sol.solve([jn.e_fermi])
    assert res.converged
    for e in (0, 1):
        rows = np.nonzero(res.energy_index == e)[0]
        n = res.n_open[e]
        assert n >= 2
        assert abs(res.G[e] - n) < G_TOL
        T = res.T[rows][:, :n]
        assert np.max(np.abs(T[np.arange(n), res.channel[rows]] - 1.0)) < G_TOL
        assert np.max(np.abs(res.R[rows][:, :n])) < G_TOL
    sol.close()


def test_reciprocity_and_lattice_shift_on_gpu():
    # T^{L->R}(kappa)[o, i] = T^{R->L}(-kappa)[i~, o~] with ~ the reversed mode: the
    # right-incident solve at kappa returns the -kappa problem in its upper slot
    from paper_1009_5300_gb300 import IOBMSolver
    jn = kb_junction()
    E = jn.e_fermi - 0.02
    k = kappa_of(jn, 0.33, 0.52)
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    sol.set_bloch(k)
    L = sol.solve([E], side=0)
    n = L.n_open[0]
    TL = np.zeros((n, n))
    for r in np.nonzero(L.energy_index == 0)[0]:
        TL[:, L.channel[r]] = L.T[r, :n]
    R = sol.solve([E], side=1)
    TRm = np.zeros((n, n))
    for r in np.nonzero(R.energy_index == 1)[0]:
        TRm[:, R.channel[r]] = R.T[r, :n]
    md_p = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, 4, E, kappa=k)
    md_m = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, 4, E, kappa=(-k[0], -k[1]))
    nu_m = [tuple(md_m.nu[m]) for m in md_m.open_modes]

    def rev(a, N):
        return -a if -a in range(-(N // 2), N - N // 2) else a

    flip = [nu_m.index((rev(a, jn.nx), rev(b, jn.ny)))
            for a, b in (tuple(md_p.nu[m]) for m in md_p.open_modes)]
    for o in range(n):
        for i in range(n):
            assert abs(TL[o, i] - TRm[flip[i], flip[o]]) < G_TOL
    assert abs(L.G[0] - R.G[1]) < G_TOL
    # kappa + 2 pi / L_x: the same Bloch waves, the same conductance
    sol.set_bloch((k[0] + 2 * math.pi / (jn.nx * jn.hx), k[1]))
    assert abs(sol.solve([E]).G[0] - L.G[0]) < G_TOL
    sol.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gradient_at_kappa_matches_oracle(precision):
    from paper_1009_5300_gb300 import IOBMSolver
    jn = S.small_wire(nx=8, ny=8, nz=20, h=0.6, natom=2, spacing=3.0, depth=0.6, width=0.9,
                      rs=1.5, kb_kinds=S.SP, kb_radius=1.2, kb_width=0.5, seed=11, nf=4)
    E = jn.e_fermi
    k = kappa_of(jn, 0.35, -0.2)
    ref = transport.grad_V(jn, E, kappa=k)
    sol = IOBMSolver.from_junction(jn, precision=precision)
    sol.set_bloch(k)
    g, G = sol.grad_V(E)
    g = g.cpu().numpy()
    scale = np.max(np.abs(ref))
    print(f"{precision}: max |dg| {np.max(np.abs(g - ref)) / scale:.2e} of max |g|")
    assert abs(G - transport.conductance(jn, E, k)) < G_TOL
    assert np.max(np.abs(g - ref)) < 1e-5 * scale
    sol.close()


def test_kappa_zero_restores_the_cocg_path():
    # setting kappa back to 0 gives the periodic solve bit for bit
    from paper_1009_5300_gb300 import IOBMSolver
    jn = kb_junction()
    E = jn.e_fermi
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    a = sol.solve([E])
    sol.set_bloch(kappa_of(jn, 0.2, 0.1))
    sol.solve([E])
    sol.set_bloch((0.0, 0.0))
    b = sol.solve([E])
    assert np.array_equal(a.T, b.T) and np.array_equal(a.iterations, b.iterations)
    sol.close()


def test_kappa_needs_the_free_propagator():
    from paper_1009_5300_gb300 import IOBMSolver
    from paper_1009_5300_gb300._lib import IOBM_E_UNSUPPORTED, IOBMError
    jn = kb_junction()
    sol = IOBMSolver.from_junction(jn, precision="mixed", use_precond="eq10")
    with pytest.raises(IOBMError) as err:
        sol.set_bloch((0.1, 0.0))
    assert err.value.code == IOBM_E_UNSUPPORTED
    sol.close()
