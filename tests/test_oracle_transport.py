"""Pins for the oracle's scattering solutions, T/R/G and dG/dV (Eqs. 6-7, Sec. III)."""
import math

import numpy as np
import pytest

import iobm_synth as S
from oracle import modes, transport
from oracle.fd import second_derivative_weights


def flat_junction(nf, nx=12, ny=10, nz=14, h=0.6, rs=1.5):
    jn = S.small_wire(nx=nx, ny=ny, nz=nz, h=h, natom=1, depth=0.0, rs=rs, nf=nf)
    return jn.copy_with(V=np.zeros_like(jn.V))


@pytest.mark.parametrize("nf", [1, 2, 4])
def test_flat_potential_integer_conductance(nf):
    # constant potential: every open channel transmits fully, G = N_open G_0 exactly
    jn = flat_junction(nf)
    sol = transport.solve(jn, jn.e_fermi)
    assert sol.n_open >= 3
    assert np.max(np.abs(sol.T - np.eye(sol.n_open))) < 1e-10
    assert np.max(np.abs(sol.R)) < 1e-10
    assert abs(sol.G - sol.n_open) < 1e-10


def transfer_T_nf1(V, E_mode, h):
    """psi on planes -1 .. n (transition planes 0..n-1), transmitted wave lam^k beyond."""
    n = len(V)
    kh = math.acos(1 - h * h * E_mode)
    lam = complex(math.cos(kh), math.sin(kh))
    psi = {n: lam ** n, n + 1: lam ** (n + 1)}   # electrode planes n, n+1 (plane index)
    # row k (k = n .. 0): psi_{k-1} = 2 h^2 (E - V_k) ... solved for psi_{k-1}
    for k in range(n, -1, -1):
        Vk = V[k] if k < n else 0.0
        psi[k - 1] = -2 * h * h * (E_mode - Vk) * psi[k] + 2 * psi[k] - psi[k + 1]
    # on planes -1, 0 the wave is a lam^k + b lam^-k
    M = np.array([[lam ** -1, lam], [1.0, 1.0]])
    a, b = np.linalg.solve(M, np.array([psi[-1], psi[0]]))
    t = 1.0 / a
    r = b / a
    return abs(t) ** 2, abs(r) ** 2


def test_uniform_vz_nf1_transfer_matrix():
    # laterally uniform V(z): the lateral modes decouple and each channel is a
    # 1D chain at energy E - eps_perp(nu)
    nx, ny, nz, h = 10, 9, 30, 0.5
    jn = S.small_wire(nx=nx, ny=ny, nz=nz, h=h, natom=1, depth=0.0, rs=1.2, nf=1)
    z = np.arange(nz) * h
    Vz = 0.35 * np.exp(-((z - 7.0) / 1.3) ** 2) - 0.2 * np.exp(-((z - 9.5) / 0.8) ** 2)
    jn = jn.copy_with(V=np.broadcast_to(Vz[:, None, None], (nz, ny, nx)).copy())
    E = jn.e_fermi
    sol = transport.solve(jn, E)
    md = sol.md
    assert sol.n_open >= 2
    for i, m in enumerate(sol.open_modes):
        Tm, Rm = transfer_T_nf1(Vz, E - md.eps_perp[m], h)
        assert abs(sol.T[i, i] - Tm) < 1e-10
        assert abs(sol.R[i, i] - Rm) < 1e-10
        off = np.delete(sol.T[:, i], i)
        assert np.max(np.abs(off)) < 1e-12 if len(off) else True


def poschl_teller_T(k, V0, a):
    """Continuum transmission through V0 / cosh^2(z/a) (hbar = m = 1), textbook closed form."""
    s = math.sinh(math.pi * k * a) ** 2
    q = 8 * V0 * a * a - 1
    c = math.cosh(0.5 * math.pi * math.sqrt(q)) ** 2 if q > 0 else math.cos(0.5 * math.pi * math.sqrt(-q)) ** 2
    return s / (s + c)


@pytest.mark.parametrize("nf,h,tol", [(4, 0.25, 2e-5), (1, 0.1, 4e-3)])
def test_uniform_vz_poschl_teller(nf, h, tol):
    # laterally uniform sech^2 barrier: the (0,0) channel matches the continuum
    # closed form up to the FD error (O(h^(2 N_f)))
    V0, a = 0.2, 1.5
    Lz = 48.0
    nz = int(round(Lz / h))
    jn = S.small_wire(nx=3, ny=3, nz=nz, h=h, natom=1, depth=0.0, rs=3.0, nf=nf)
    z = (np.arange(nz) - 0.5 * (nz - 1)) * h
    Vz = V0 / np.cosh(z / a) ** 2
    jn = jn.copy_with(V=np.broadcast_to(Vz[:, None, None], (nz, 3, 3)).copy())
    E = 0.18
    sol = transport.solve(jn, E)
    assert sol.n_open == 1
    k = math.sqrt(2 * E)
    assert abs(sol.T[0, 0] - poschl_teller_T(k, V0, a)) < tol


def kb_junction(nf=4):
    return S.small_wire(nx=12, ny=12, nz=26, h=0.5, natom=2, spacing=3.4, depth=0.7, width=0.9,
                        rs=1.6, kb_kinds=S.SP, nf=nf, seed=77)


@pytest.mark.parametrize("nf", [1, 4])
def test_current_conservation(nf):
    jn = kb_junction(nf)
    sol = transport.solve(jn, jn.e_fermi)
    assert sol.n_open >= 3
    per_in = sol.T.sum(axis=0) + sol.R.sum(axis=0)
    assert np.max(np.abs(per_in - 1.0)) < 1e-10
    assert abs(sol.G + sol.R.sum() - sol.n_open) < 1e-10


def test_reciprocity():
    jn = kb_junction(4)
    E = jn.e_fermi - 0.02
    L = transport.solve(jn, E, side="L")
    R = transport.solve(jn, E, side="R")
    # time reversal maps lateral mode nu to -nu, so S = S^T reads
    # T^{L->R}[o, i] = T^{R->L}[-i, -o] (kappa = 0, real V and KB)
    nu = [tuple(L.md.nu[m]) for m in L.open_modes]
    flip = [nu.index((-a if -a in range(-(jn.nx // 2), jn.nx - jn.nx // 2) else a,
                      -b if -b in range(-(jn.ny // 2), jn.ny - jn.ny // 2) else b)) for a, b in nu]
    n = L.n_open
    for o in range(n):
        for i in range(n):
            assert abs(L.T[o, i] - R.T[flip[i], flip[o]]) < 1e-10
    assert abs(L.G - R.G) < 1e-10


def test_gradient_matches_finite_differences():
    jn = S.small_wire(nx=8, ny=8, nz=20, h=0.6, natom=2, spacing=3.0, depth=0.6, width=0.9,
                      rs=1.4, kb_kinds=S.SP, nf=4, seed=5)
    assert modes.count_open_channels(8, 8, 0.6, 0.6, 0.6, 4, jn.e_fermi) >= 3
    E = jn.e_fermi
    g = transport.grad_V(jn, E)
    rng = np.random.default_rng(1)
    pts = [tuple(rng.integers(0, s) for s in jn.V.shape) for _ in range(6)]
    pts.append((0, 2, 2))                   # an end plane (inside the self-energy rows)
    dV = 1e-5
    for p in pts:
        Vp = jn.V.copy(); Vp[p] += dV
        Vm = jn.V.copy(); Vm[p] -= dV
        fd = (transport.conductance(jn.copy_with(V=Vp), E)
              - transport.conductance(jn.copy_with(V=Vm), E)) / (2 * dV)
        assert abs(fd - g[p]) < 1e-6 * max(1.0, abs(g).max()), (p, fd, g[p])


def test_gradient_zero_for_flat_potential():
    # at V = const every channel transmits fully and r = 0, so dG/dV = 0
    jn = flat_junction(4)
    g = transport.grad_V(jn, jn.e_fermi)
    assert np.max(np.abs(g)) < 1e-9


def test_eigenchannels_flat_and_uniform():
    # flat potential: every eigenchannel transmits fully
    jn = flat_junction(4)
    tau = transport.eigenchannels(transport.solve(jn, jn.e_fermi))
    assert np.max(np.abs(tau - 1.0)) < 1e-10
    # laterally uniform V(z): the channels decouple, T is diagonal, and the
    # eigenchannel transmissions are its diagonal (each from the 1D transfer matrix)
    nx, ny, nz, h = 10, 9, 30, 0.5
    jn = S.small_wire(nx=nx, ny=ny, nz=nz, h=h, natom=1, depth=0.0, rs=1.2, nf=1)
    z = np.arange(nz) * h
    Vz = 0.35 * np.exp(-((z - 7.0) / 1.3) ** 2) - 0.2 * np.exp(-((z - 9.5) / 0.8) ** 2)
    jn = jn.copy_with(V=np.broadcast_to(Vz[:, None, None], (nz, ny, nx)).copy())
    sol = transport.solve(jn, jn.e_fermi)
    tau = transport.eigenchannels(sol)
    ref = np.sort([transfer_T_nf1(Vz, jn.e_fermi - sol.md.eps_perp[m], h)[0] for m in sol.open_modes])[::-1]
    assert np.max(np.abs(tau - ref)) < 1e-10


def test_eigenchannels_bounds_and_sum():
    # unitarity (T + R = 1 per channel, t~^H t~ + r~^H r~ = 1) puts every eigenvalue
    # in [0, 1]; the trace of t~^H t~ is G
    jn = kb_junction(4)
    sol = transport.solve(jn, jn.e_fermi)
    tau = transport.eigenchannels(sol)
    assert len(tau) == sol.n_open
    assert np.all(tau > -1e-12) and np.all(tau < 1 + 1e-10)
    assert abs(tau.sum() - sol.G) < 1e-10
    assert np.all(np.diff(tau) <= 1e-15)
