"""Iterative FP64 oracle for grids whose assembled operator cannot be factored.

Test infrastructure only, like the rest of ``oracle/``: it shares no code with
the CUDA path and the library never imports it.

At the benchmark sizes (48 x 48 x 160 and up) the dense end blocks of Eq. 8
alone hold (N_f N_xy)^2 entries per end, so ``transport.solve`` (sparse LU of
the assembled matrix) is out of reach.  This module reaches the same exact
solution of Eq. 7 by a different route:

* the operator is ``operator.apply_A`` (E - H_T - H~ applied matrix-free, the
  self-energy through the explicit sums of Eqs. 18-1/19; pinned equal to the
  assembled matrix in tests/test_oracle_operator.py);
* the linear solve is restarted GMRES (scipy), FP64 complex, followed by
  iterative refinement on the true residual b - A psi until
  ||b - A psi||_2 / ||b||_2 <= tol (1e-12 by default), so the answer does not
  depend on how scipy measures convergence;
* GMRES is preconditioned by the free propagator (E - T - H~)^{-1}, written
  here in its own form: the lateral Fourier transform of Eq. 19 (numpy FFT
  with the bin of mode nu at nu mod N) makes the potential-free operator
  block diagonal, one banded N_z x N_z system per lateral mode with diagonal
  E - eps_perp(nu) + w_0 / (2 h_z^2), off-diagonals w_n / (2 h_z^2) and the
  per-mode self-energy Sigma~_nu (Eq. 18-2 generalised to N_f planes) on the
  N_f outermost planes at each end; each system is solved by banded LU
  (scipy.linalg.solve_banded).  The preconditioner only changes how fast GMRES
  converges, never the answer, which is checked against ``apply_A``;
* the solved waves are projected with ``transport.project`` (Eq. 6 with the
  explicit Eq. 19 sums) and T, R, G formed as in ``transport.solve``.

Pinned by (tests/test_oracle_iterative.py): the banded per-mode propagator
equals ``operator.free_inverse`` (sparse LU of the assembled potential-free
matrix) on small grids, at kappa = 0 and kappa != 0; ``solve_gmres`` equals the
sparse-LU ``transport.solve`` (t, r, T, R, G) on a small junction with s/p
projectors, for left and right incidence; the flat-potential junction gives
T = identity and G = N_open.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .modes import ModeData
from .operator import apply_A, end_planes
from .transport import Solution, modes_for, project, source_vector


def _fft_bins(jn, md: ModeData):
    """FFT bin (ky, kx) of every mode: exp(-i G_nu . r) with G_nu = 2 pi nu / L is the
    DFT kernel at frequency nu mod N."""
    return md.nu[:, 1] % jn.ny, md.nu[:, 0] % jn.nx


def _gauge(jn, md: ModeData):
    """exp(-i kappa . r_l) on the lateral plane, or None at kappa = 0."""
    if md.kappa[0] == 0.0 and md.kappa[1] == 0.0:
        return None
    x = np.arange(jn.nx) * jn.hx
    y = np.arange(jn.ny) * jn.hy
    return np.exp(-1j * (md.kappa[1] * y[:, None] + md.kappa[0] * x[None, :]))


def banded_mode_systems(jn, E: float, md: ModeData) -> np.ndarray:
    """Per lateral mode the N_z x N_z matrix of E - T - H~ in LAPACK banded storage:
    ab[m, N_f + i - j, j] = A_m[i, j] (plane indices i, j)."""
    nf, nz = jn.nf, jn.nz
    w = md.w
    nm = len(md.nu)
    ab = np.zeros((nm, 2 * nf + 1, nz), dtype=np.complex128)
    # kinetic z part + (E - eps_perp) on the diagonal
    ab[:, nf, :] = (E - md.eps_perp)[:, None] + 0.5 * w[0] / jn.hz ** 2
    for n in range(1, nf + 1):
        c = 0.5 * w[n] / jn.hz ** 2
        ab[:, nf - n, n:] = c          # A[i, i + n]: row i = j - n
        ab[:, nf + n, : nz - n] = c    # A[i, i - n]: row i = j + n
    # self-energy blocks on the N_f outermost planes (depth d counted inward)
    for d in range(nf):
        for e in range(nf):
            s = md.sigma[:, d, e]
            ab[:, nf + d - e, e] -= s                     # left end: planes d, e
            ab[:, nf + e - d, nz - 1 - e] -= s            # right end: planes nz-1-d, nz-1-e
    return ab


class FreePropagator:
    """z = (E - T - H~)^{-1} r by lateral FFT and per-mode banded solves."""

    def __init__(self, jn, E: float, md: ModeData):
        self.jn, self.md = jn, md
        self.ab = banded_mode_systems(jn, E, md)
        self.ky, self.kx = _fft_bins(jn, md)
        self.gauge = _gauge(jn, md)

    def __call__(self, r: np.ndarray) -> np.ndarray:
        jn, nf = self.jn, self.jn.nf
        nxy = jn.nx * jn.ny
        v = np.asarray(r, dtype=np.complex128).reshape(jn.nz, jn.ny, jn.nx)
        if self.gauge is not None:
            v = v * self.gauge[None]
        spec = np.fft.fft2(v, axes=(1, 2)) / nxy           # Eq. 19 per plane
        modes = spec[:, self.ky, self.kx]                   # [z][mode]
        out = np.empty_like(modes)
        for m in range(modes.shape[1]):
            out[:, m] = sla.solve_banded((nf, nf), self.ab[m], modes[:, m])
        Y = np.zeros_like(spec)
        Y[:, self.ky, self.kx] = out
        z = np.fft.ifft2(Y, axes=(1, 2)) * nxy
        if self.gauge is not None:
            z = z * np.conj(self.gauge)[None]
        return z


def free_propagator_modes(jn, E: float, md: ModeData, r: np.ndarray) -> np.ndarray:
    """(E - T - H~)^{-1} r for one vector r [nz][ny][nx] (see FreePropagator)."""
    return FreePropagator(jn, E, md)(r)


@dataclasses.dataclass
class IterativeSolution(Solution):
    residuals: np.ndarray = None     # ||b - A psi|| / ||b|| per incident channel
    gmres_iterations: np.ndarray = None


def gmres_wave(jn, E: float, md: ModeData, b: np.ndarray, M: FreePropagator, tol: float = 1e-12,
               restart: int = 80, max_outer: int = 20):
    """psi with ||b - A psi|| <= tol ||b|| (restarted GMRES + refinement on the true residual).
    Returns (psi, relative residual, total GMRES matrix-vector products)."""
    shape = (jn.nz, jn.ny, jn.nx)
    n = jn.npts
    A = spla.LinearOperator((n, n), dtype=np.complex128,
                            matvec=lambda v: apply_A(jn, E, md, v.reshape(shape)).reshape(-1))
    P = spla.LinearOperator((n, n), dtype=np.complex128,
                            matvec=lambda v: M(v).reshape(-1))
    bf = b.reshape(-1).astype(np.complex128)
    nb = np.linalg.norm(bf)
    x = np.zeros(n, dtype=np.complex128)
    r = bf.copy()
    count = [0]

    def cb(_):
        count[0] += 1

    res = 1.0
    for _ in range(max_outer):
        # the correction equation A d = r to a loose relative tolerance; the true
        # residual below decides when to stop
        d, _info = spla.gmres(A, r, rtol=1e-6, atol=0.0, restart=restart, maxiter=20, M=P,
                              callback=cb, callback_type="pr_norm")
        x = x + d
        r = bf - A.matvec(x)
        res = np.linalg.norm(r) / nb
        if res <= tol:
            break
    return x.reshape(shape), float(res), count[0]


def solve_gmres(jn, E: float, side: str = "L", channels: Optional[Sequence[int]] = None,
                tol: float = 1e-12, kappa=(0.0, 0.0)) -> IterativeSolution:
    """Eq. 7 for every open incident channel (or the subset `channels`) by
    preconditioned GMRES to tol; projection, T, R and G as in transport.solve."""
    md = modes_for(jn, E, kappa)
    opens = md.open_modes
    chan = list(range(len(opens))) if channels is None else list(channels)
    M = FreePropagator(jn, E, md)
    psis, ts, rs, res, its = [], [], [], [], []
    for c in chan:
        m = opens[c]
        b = source_vector(jn, md, m, side, matrix_free=True)
        psi, rr, k = gmres_wave(jn, E, md, b, M, tol=tol)
        t, r = project(jn, md, psi, m, side)
        psis.append(psi)
        ts.append(t)
        rs.append(r)
        res.append(rr)
        its.append(k)
    vel = md.vel[opens]
    t = np.array(ts).T if ts else np.zeros((len(opens), 0), np.complex128)
    r = np.array(rs).T if rs else np.zeros((len(opens), 0), np.complex128)
    vin = vel[chan] if chan else np.zeros(0)
    T = np.abs(t) ** 2 * vel[:, None] / vin[None, :]
    R = np.abs(r) ** 2 * vel[:, None] / vin[None, :]
    return IterativeSolution(
        E=E, side=side, md=md, open_modes=opens,
        psi=np.array(psis) if psis else np.zeros((0,) + (jn.nz, jn.ny, jn.nx), np.complex128),
        t=t, r=r, T=T, R=R, G=float(T.sum()), vel=vel,
        residuals=np.array(res), gmres_iterations=np.array(its))
