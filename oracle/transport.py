"""Exact scattering solutions, channel projection, conductance and dG/dV (FP64).

Paper passages followed:

* Eq. 7: one linear solve of (E - H_T - H~) Psi = b per incident wave; here by
  sparse LU (SuperLU through scipy) of the assembled matrix, i.e. the exact
  solution of the equations the iterative method converges to.  The KB term
  enters through the equivalent augmented system built in ``operator``.
* The source b (Eq. 7, N_f planes): the FD couplings of the first N_f transition
  rows to the electrode planes applied to the incident wave there, plus the
  real-space self-energy block (Eq. 8) applied to the incident wave on the
  first N_f planes, both with a minus sign.  Built in real space.
* Eq. 6: beyond the exit end the wave is sum_i t_i Phi^tra_i, before the entry
  end Phi^in + sum_i r_i Phi^ref_i.  On the N_f outermost transition planes of
  each end the wave already has this Bloch form (the electrode rows reach
  them), so per lateral mode (Eq. 19, explicit sum) the N_f coefficients follow
  from an N_f x N_f solve with Q_in; the propagating one is t (or r).
* Landauer-Buttiker (Sec. III): G = G_0 sum_{o,i} T_oi with
  T_oi = |t_oi|^2 v_o / v_i (flux normalisation by the discrete group velocity)
  and R_oi = |r_oi|^2 v_o / v_i.
* Eigenchannels (Sec. IV, Table II): eigenvalues of T^dagger T for the
  flux-normalised transmission matrix.
* dG/dV(r) (not in the paper; follows from Eq. 7 with dA/dV(r) = -e_r e_r^T and
  A = A^T): with A lambda_o = w_o, where w_o is the linear functional that
  returns t_o from a solved wave,
  dG/dV(r) = sum_{o,i} 2 (v_o / v_i) Re[conj(t_oi) lambda_o(r) psi_i(r)].

Pinned by: flat potential gives T = identity and G = N_open exactly; laterally
uniform V(z) against an independent 1D transfer matrix; T + R = N_open per
incident channel; reciprocity T^{LR} = (T^{RL})^T; gradient against central
finite differences and zero at V = 0; tests/test_oracle_transport.py.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, Optional, Sequence

import numpy as np
import scipy.sparse.linalg as spla

from .modes import ModeData, mode_data, lateral_phase
from .operator import assemble_augmented, sigma_dense, end_planes, kb_factors


@dataclasses.dataclass
class Solution:
    E: float
    side: str                      # incident side 'L' or 'R'
    md: ModeData
    open_modes: np.ndarray         # mode indices of the open channels (canonical order)
    psi: np.ndarray                # [n_in][nz][ny][nx] complex
    t: np.ndarray                  # [n_out][n_in]
    r: np.ndarray                  # [n_out][n_in]
    T: np.ndarray                  # [n_out][n_in]
    R: np.ndarray                  # [n_out][n_in]
    G: float                       # units of G_0
    vel: np.ndarray                # [n_open]

    @property
    def n_open(self) -> int:
        return len(self.open_modes)


def modes_for(jn, E: float, kappa=(0.0, 0.0)) -> ModeData:
    return mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, jn.nf, E, kappa=kappa)


def incident_wave_planes(jn, md: ModeData, m: int, depths: np.ndarray) -> np.ndarray:
    """Unit incident wave of mode m at depth index d (negative = electrode plane -d):
    f(l) lambda_in^d with f(l) = exp(i (G_m + kappa) . r_l); returned as [len(depths)][N_xy]."""
    lam = md.lam[m, md.prop[m]]
    # the row of mode m of the Eq. 19 phase matrix, conjugated: exp(+i (G_m + kappa) . r_l)
    x = np.arange(jn.nx) * jn.hx
    y = np.arange(jn.ny) * jn.hy
    Gx = 2.0 * np.pi * md.nu[m, 0] / (jn.nx * jn.hx) + md.kappa[0]
    Gy = 2.0 * np.pi * md.nu[m, 1] / (jn.ny * jn.hy) + md.kappa[1]
    f = np.exp(1j * (Gy * y[:, None] + Gx * x[None, :])).reshape(-1)
    return (lam ** depths)[:, None] * f[None, :]


def source_vector(jn, md: ModeData, m: int, side: str, S: Optional[np.ndarray] = None,
                  matrix_free: bool = False) -> np.ndarray:
    """b for a unit incident wave in mode m from side 'L' or 'R' (Eq. 7).  With
    matrix_free the self-energy term goes through the explicit Eq. 19 sums instead of
    the dense Eq. 8 block (for lateral grids whose dense block does not fit)."""
    from .operator import _sigma_apply_end
    nf = jn.nf
    nxy = jn.nx * jn.ny
    K = md.K
    d = np.arange(nf)
    phi_in = incident_wave_planes(jn, md, m, d)                  # transition planes, depth d
    phi_el = incident_wave_planes(jn, md, m, -(d + 1))            # electrode planes e = 1..nf
    coupling = K @ phi_el                                         # [d][l]
    if matrix_free:
        sig = _sigma_apply_end(jn, md, phi_in)
    else:
        if S is None:
            S = sigma_dense(jn, md)
        sig = (S @ phi_in.reshape(-1)).reshape(nf, nxy)
    bplanes = -coupling - sig
    b = np.zeros((jn.nz, nxy), dtype=np.complex128)
    b[end_planes(jn, side)] = bplanes
    return b.reshape(jn.nz, jn.ny, jn.nx)


def _coefficients(jn, md: ModeData, planes_vals: np.ndarray) -> np.ndarray:
    """Per mode, solve Q_in a = psi~ over the N_f end planes; return a [mode][root]."""
    nxy = jn.nx * jn.ny
    F = lateral_phase(jn.nx, jn.ny, jn.hx, jn.hy, md)
    ft = (F @ planes_vals.T) / nxy                  # [mode][d]  (Eq. 19)
    d = np.arange(md.nf)
    a = np.zeros_like(ft)
    for m in range(len(md.nu)):
        Qin = md.lam[m][None, :] ** (-d[:, None])
        a[m] = np.linalg.solve(Qin, ft[m])
    return a


def project(jn, md: ModeData, psi: np.ndarray, m_in: int, side: str):
    """(t, r) over the open modes for one solved wave psi [nz][ny][nx] (Eq. 6)."""
    nxy = jn.nx * jn.ny
    exit_side = "R" if side == "L" else "L"
    flat = psi.reshape(jn.nz, nxy)
    opens = md.open_modes
    a_exit = _coefficients(jn, md, flat[end_planes(jn, exit_side)])
    entry = flat[end_planes(jn, side)].copy()
    entry -= incident_wave_planes(jn, md, m_in, np.arange(jn.nf))
    a_entry = _coefficients(jn, md, entry)
    t = np.array([a_exit[m, md.prop[m]] for m in opens])
    r = np.array([a_entry[m, md.prop[m]] for m in opens])
    return t, r


def solve(jn, E: float, side: str = "L", channels: Optional[Sequence[int]] = None,
          kappa=(0.0, 0.0)) -> Solution:
    """Exact solve of Eq. 7 for every open incident channel (or the given subset,
    indices into the open-channel list), at lateral Bloch vector kappa."""
    md = modes_for(jn, E, kappa)
    opens = md.open_modes
    chan = list(range(len(opens))) if channels is None else list(channels)
    M = assemble_augmented(jn, E, md)
    lu = spla.splu(M)
    S = sigma_dense(jn, md)
    nproj = len(jn.projectors)
    psis, ts, rs = [], [], []
    for c in chan:
        m = opens[c]
        b = source_vector(jn, md, m, side, S).reshape(-1)
        rhs = np.concatenate([b, np.zeros(nproj, np.complex128)])
        x = lu.solve(rhs)[: jn.npts].reshape(jn.nz, jn.ny, jn.nx)
        t, r = project(jn, md, x, m, side)
        psis.append(x)
        ts.append(t)
        rs.append(r)
    vel = md.vel[opens]
    t = np.array(ts).T if ts else np.zeros((len(opens), 0), np.complex128)
    r = np.array(rs).T if rs else np.zeros((len(opens), 0), np.complex128)
    vin = vel[chan] if chan else np.zeros(0)
    T = np.abs(t) ** 2 * vel[:, None] / vin[None, :]
    R = np.abs(r) ** 2 * vel[:, None] / vin[None, :]
    return Solution(E=E, side=side, md=md, open_modes=opens,
                    psi=np.array(psis) if psis else np.zeros((0, jn.nz, jn.ny, jn.nx), np.complex128),
                    t=t, r=r, T=T, R=R, G=float(T.sum()), vel=vel)


def conductance(jn, E: float, kappa=(0.0, 0.0)) -> float:
    return solve(jn, E, kappa=kappa).G


def eigenchannels(sol: Solution) -> np.ndarray:
    """Eigenchannel transmissions (Sec. IV, Table II: eigenvalues of T^dagger T, T the
    transmission matrix) of a solve over every open incident channel: with the
    flux-normalised amplitudes t~_oi = t_oi sqrt(v_o / v_i), the eigenvalues of
    t~^H t~ in descending order."""
    if sol.t.shape[1] != sol.n_open:
        raise ValueError("eigenchannels need every open incident channel")
    v = sol.vel
    tt = sol.t * np.sqrt(v[:, None] / v[None, :])
    return np.sort(np.linalg.eigvalsh(tt.conj().T @ tt))[::-1]


def exit_functional(jn, md: ModeData, m_out: int, side: str = "L") -> np.ndarray:
    """w_o with t_o = w_o^T psi (unconjugated), supported on the exit planes."""
    nxy = jn.nx * jn.ny
    exit_side = "R" if side == "L" else "L"
    F = lateral_phase(jn.nx, jn.ny, jn.hx, jn.hy, md)
    d = np.arange(md.nf)
    Qin = md.lam[m_out][None, :] ** (-d[:, None])
    row = np.linalg.inv(Qin)[md.prop[m_out]]           # [d]
    wv = np.zeros((jn.nz, nxy), dtype=np.complex128)
    wv[end_planes(jn, exit_side)] = row[:, None] * F[m_out][None, :] / nxy
    return wv.reshape(jn.nz, jn.ny, jn.nx)


def grad_V(jn, E: float, sol: Optional[Solution] = None, kappa=(0.0, 0.0)) -> np.ndarray:
    """dG/dV(r) in G_0 per Ha for left-incident waves: lambda_o = A^{-T} w_o (the
    same operator at kappa = 0, where A = A^T; the transposed solve otherwise)."""
    if sol is None:
        sol = solve(jn, E, kappa=kappa)
    md = sol.md
    M = assemble_augmented(jn, E, md)
    lu = spla.splu(M)
    trans = "N" if (md.kappa[0] == 0.0 and md.kappa[1] == 0.0) else "T"
    nproj = len(jn.projectors)
    opens = sol.open_modes
    g = np.zeros((jn.nz, jn.ny, jn.nx))
    for o, m_out in enumerate(opens):
        wv = exit_functional(jn, md, m_out, sol.side).reshape(-1)
        lam_o = lu.solve(np.concatenate([wv, np.zeros(nproj, np.complex128)]), trans=trans)[: jn.npts]
        lam_o = lam_o.reshape(jn.nz, jn.ny, jn.nx)
        for i in range(sol.psi.shape[0]):
            coef = 2.0 * sol.vel[o] / sol.vel[i] * np.conj(sol.t[o, i])
            g += np.real(coef * lam_o * sol.psi[i])
    return g


def residual(jn, E: float, md: ModeData, psi: np.ndarray, b: np.ndarray) -> float:
    """||b - A psi||_2 / ||b||_2 with the matrix-free FP64 operator."""
    from .operator import apply_A
    r = b - apply_A(jn, E, md, psi)
    return float(np.linalg.norm(r) / np.linalg.norm(b))
