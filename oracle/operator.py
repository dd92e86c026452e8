"""The truncated IOBM operator E - H_T - H~ and the preconditioner (FP64, CPU).

Paper passages followed:

* Eq. 1: the kinetic operator -1/2 d^2/dr^2 with FD weights on each axis;
  x and y periodic (Sec. II takes both lateral directions periodic), or Bloch
  periodic psi(r + L) = exp(i kappa L) psi(r) for a lateral Bloch vector kappa
  (Eq. 8): a coupling that wraps across the lateral period carries that phase.
* Eqs. 2-4: H_T is the Hamiltonian of planes z_0 .. z_{N_z+1}; couplings that
  would reach beyond those planes are dropped from H_T (they are accounted for
  by the self-energy and the source).  H_T contains the local potential V(r)
  and the nonlocal Kleinman-Bylander term sum_p E_p |p><p| (the norm-conserving
  pseudopotentials of Sec. III), with <p|psi> = h_x h_y h_z sum_r p(r) psi(r).
* Eqs. 7 and 7-2: the solved matrix is E - H_T - H~, with H~ holding the
  self-energy blocks on the N_f outermost planes at each end (one plane,
  z_0 and z_{N_z+1}, for N_f = 1).
* Eq. 8: the real-space self-energy block,
  Sigma_{(d,l),(d',l')} = (1/N_xy) sum_nu exp(i G_nu . (r_l - r_l')) Sigma~_nu[d, d'],
  built here as an explicit dense sum (no FFT).
* Eq. 10: the preconditioner P gamma(r) = C_0 gamma(r) + C_1 sum over the six
  face neighbours r +- h_x, r +- h_y, r +- h_z, with C_0 = 1 and
  C_1 = exp(-alpha) (Sec. III); laterally periodic, zero beyond the end planes.

`apply_A` is the same operator applied matrix-free, with the self-energy
applied through the explicit lateral Fourier sums of Eqs. 18-1/19 (dense DFT
matrices, not an FFT) so that it also works at sizes where the dense
real-space blocks do not fit.

`free_inverse` applies (E - T - H~)^{-1}, the Green's function of the transition
region with the potential removed (the quantity the paper's preconditioner of
Eq. 10 approximates by a truncated Laplacian Green's function), by sparse LU of
the assembled matrix.

Pinned by: A == A^T exactly; the dense Eq. 8 block equals the Appendix
surface Green's function (Eq. A-10) for N_f = 1; matrix-free and assembled forms
agree; P's symbol bound (Sec. III, alpha > ln 6); tests/test_oracle_operator.py.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fd import second_derivative_weights
from .modes import ModeData, lateral_phase


def _fd_matrix_periodic(n: int, w: np.ndarray, phase=None) -> sp.csr_matrix:
    """n x n circulant matrix of the FD second-derivative weights (dimensionless).
    With phase = exp(i kappa L): Bloch-periodic, a coupling to i + s >= n carries
    phase and one to i + s < 0 its conjugate."""
    nf = len(w) - 1
    rows, cols, vals = [], [], []
    for i in range(n):
        for s in range(-nf, nf + 1):
            rows.append(i)
            cols.append((i + s) % n)
            v = w[abs(s)]
            if phase is not None:
                v = v * (phase if i + s >= n else (np.conj(phase) if i + s < 0 else 1.0))
            vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))  # duplicates summed


def _fd_matrix_truncated(n: int, w: np.ndarray) -> sp.csr_matrix:
    """n x n banded FD matrix with the terms beyond the ends dropped (Eq. 4)."""
    nf = len(w) - 1
    rows, cols, vals = [], [], []
    for i in range(n):
        for s in range(-nf, nf + 1):
            j = i + s
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
                vals.append(w[abs(s)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def _bloch_phases(jn, kappa):
    """(exp(i kappa_x L_x), exp(i kappa_y L_y)), or (None, None) at kappa = 0."""
    if kappa[0] == 0.0 and kappa[1] == 0.0:
        return None, None
    return (np.exp(1j * kappa[0] * jn.nx * jn.hx), np.exp(1j * kappa[1] * jn.ny * jn.hy))


def h_local(jn, kappa=(0.0, 0.0)) -> sp.csr_matrix:
    """H_T without the KB term: -1/2 (D_xx + D_yy + D_zz) + V (Eqs. 1-4), laterally
    Bloch periodic with vector kappa."""
    w = second_derivative_weights(jn.nf)
    Ix, Iy, Iz = sp.identity(jn.nx), sp.identity(jn.ny), sp.identity(jn.nz)
    px, py = _bloch_phases(jn, kappa)
    Dx = _fd_matrix_periodic(jn.nx, w, px) / jn.hx ** 2
    Dy = _fd_matrix_periodic(jn.ny, w, py) / jn.hy ** 2
    Dz = _fd_matrix_truncated(jn.nz, w) / jn.hz ** 2
    lap = (sp.kron(sp.kron(Iz, Iy), Dx) + sp.kron(sp.kron(Iz, Dy), Ix)
           + sp.kron(sp.kron(Dz, Iy), Ix))
    return (-0.5 * lap + sp.diags(jn.V.reshape(-1))).tocsr()


def kb_factors(jn):
    """(P, coupling, dvol): P is npts x nproj with P[r, p] = p(r)."""
    npts = jn.npts
    cols, rows, vals = [], [], []
    for c, p in enumerate(jn.projectors):
        rows.append(p.idx.astype(np.int64))
        cols.append(np.full(len(p.idx), c))
        vals.append(p.val)
    nproj = len(jn.projectors)
    if nproj == 0:
        return sp.csr_matrix((npts, 0)), np.zeros(0), jn.hx * jn.hy * jn.hz
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(npts, nproj))
    coupling = np.array([p.coupling for p in jn.projectors])
    return P, coupling, jn.hx * jn.hy * jn.hz


def sigma_dense(jn, md: ModeData) -> np.ndarray:
    """Real-space self-energy block [(d,l), (d',l')] of one end (Eq. 8 for N_f planes)."""
    nxy = jn.nx * jn.ny
    F = lateral_phase(jn.nx, jn.ny, jn.hx, jn.hy, md)     # [nu, l] = exp(-i G r_l)
    nf = md.nf
    S = np.zeros((nf * nxy, nf * nxy), dtype=np.complex128)
    for d in range(nf):
        for e in range(nf):
            # (1/N_xy) sum_nu exp(i G r_l) Sigma~_nu[d,e] exp(-i G r_l')
            S[d * nxy:(d + 1) * nxy, e * nxy:(e + 1) * nxy] = (
                (F.conj().T * md.sigma[:, d, e][None, :]) @ F) / nxy
    return S


def end_planes(jn, side: str) -> np.ndarray:
    """Plane indices of depth d = 0..N_f-1 at the left ('L') or right ('R') end."""
    d = np.arange(jn.nf)
    return d if side == "L" else jn.nz - 1 - d


def assemble_A_local(jn, E: float, md: ModeData) -> sp.csc_matrix:
    """E - H_T(local) - H~ as a sparse matrix with the two dense end blocks (Eqs. 7, 7-2, 8)."""
    nxy = jn.nx * jn.ny
    npts = jn.npts
    A = (E * sp.identity(npts) - h_local(jn, md.kappa)).tocoo()
    S = sigma_dense(jn, md)
    rows, cols, vals = [A.row], [A.col], [A.data.astype(np.complex128)]
    for side in ("L", "R"):
        planes = end_planes(jn, side)
        gidx = (planes[:, None] * nxy + np.arange(nxy)[None, :]).reshape(-1)
        rr, cc = np.meshgrid(gidx, gidx, indexing="ij")
        rows.append(rr.reshape(-1))
        cols.append(cc.reshape(-1))
        vals.append(-S.reshape(-1))
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(npts, npts))


def assemble_augmented(jn, E: float, md: ModeData) -> sp.csc_matrix:
    """[[A_loc, -P diag(E_p)], [dvol P^T, -I]]: eliminating the second block row
    gives back A = A_loc - dvol P diag(E_p) P^T (the KB term of H_T)."""
    A_loc = assemble_A_local(jn, E, md)
    P, coupling, dvol = kb_factors(jn)
    if P.shape[1] == 0:
        return A_loc
    nproj = P.shape[1]
    top = sp.hstack([A_loc, -P @ sp.diags(coupling)])
    bot = sp.hstack([dvol * P.T, -sp.identity(nproj)])
    return sp.vstack([top, bot]).tocsc().astype(np.complex128)


# lateral planes above this many points use numpy's FFT for the sums of Eq. 19
# (the explicit phase matrix would hold N_xy^2 entries)
EXPLICIT_DFT_LIMIT = 4096


def _sigma_apply_end(jn, md: ModeData, planes_vals: np.ndarray) -> np.ndarray:
    """Sigma applied to the N_f end planes [d][l] through Eqs. 19, 18-2 (explicit DFT;
    for planes above EXPLICIT_DFT_LIMIT points the same sums by FFT)."""
    nxy = jn.nx * jn.ny
    if nxy > EXPLICIT_DFT_LIMIT:
        return _sigma_apply_end_fft(jn, md, planes_vals)
    F = lateral_phase(jn.nx, jn.ny, jn.hx, jn.hy, md)
    ft = (F @ planes_vals.T) / nxy                    # [nu, d]  (Eq. 19)
    y = np.einsum("mde,me->md", md.sigma, ft)          # Sigma~ psi~
    return (F.conj().T @ y).T                          # back to real space [d][l]


def _sigma_apply_end_fft(jn, md: ModeData, planes_vals: np.ndarray) -> np.ndarray:
    """The sums of Eq. 19 by numpy's FFT: exp(-i G_nu . r_l) with G = 2 pi nu / L is the
    DFT kernel at frequency index nu mod N, so psi~_nu = fft2(plane)[nu_y mod N_y,
    nu_x mod N_x] / N_xy and the back sum is N_xy ifft2."""
    nf, nxy = planes_vals.shape
    ny, nx = jn.ny, jn.nx
    kx = md.nu[:, 0] % nx
    ky = md.nu[:, 1] % ny
    vals = planes_vals.reshape(nf, ny, nx)
    gauge = None
    if md.kappa[0] != 0.0 or md.kappa[1] != 0.0:
        # exp(-i (G + kappa).r) = exp(-i G.r) exp(-i kappa.r): the FFT of the gauged plane
        x = np.arange(nx) * jn.hx
        y = np.arange(ny) * jn.hy
        gauge = np.exp(-1j * (md.kappa[1] * y[:, None] + md.kappa[0] * x[None, :]))
        vals = vals * gauge[None]
    spec = np.fft.fft2(vals, axes=(1, 2)) / nxy
    ft = spec[:, ky, kx].T                              # [nu, d]
    yv = np.einsum("mde,me->md", md.sigma, ft)
    Y = np.zeros((nf, ny, nx), dtype=np.complex128)
    Y[:, ky, kx] = yv.T
    out = np.fft.ifft2(Y, axes=(1, 2)) * nxy
    if gauge is not None:
        out = out * np.conj(gauge)[None]
    return out.reshape(nf, nxy)


def apply_A(jn, E: float, md: ModeData, psi: np.ndarray) -> np.ndarray:
    """(E - H_T - H~) psi, matrix-free (psi shaped [nz][ny][nx] complex)."""
    w = second_derivative_weights(jn.nf)
    nf = jn.nf
    psi = np.asarray(psi, dtype=np.complex128)
    lap = np.zeros_like(psi)
    px, py = _bloch_phases(jn, md.kappa)

    def wrap(n, size, phase):
        # Bloch factor of psi(i + n) read from the stored period: phase past the end
        i = np.arange(size)
        return np.where(i + n >= size, phase, np.where(i + n < 0, np.conj(phase), 1.0))

    for n in range(-nf, nf + 1):
        c = w[abs(n)]
        sx = np.roll(psi, -n, axis=2)
        sy = np.roll(psi, -n, axis=1)
        if px is not None:
            sx = sx * wrap(n, jn.nx, px)[None, None, :]
            sy = sy * wrap(n, jn.ny, py)[None, :, None]
        lap += c / jn.hx ** 2 * sx
        lap += c / jn.hy ** 2 * sy
        sh = np.zeros_like(psi)
        if n >= 0:
            sh[: jn.nz - n] = psi[n:]
        else:
            sh[-n:] = psi[: jn.nz + n]
        lap += c / jn.hz ** 2 * sh
    out = E * psi + 0.5 * lap - jn.V * psi
    P, coupling, dvol = kb_factors(jn)
    if P.shape[1]:
        flat = psi.reshape(-1)
        s = dvol * (P.T @ flat)
        out = out - (P @ (coupling * s)).reshape(psi.shape)
    nxy = jn.nx * jn.ny
    for side in ("L", "R"):
        planes = end_planes(jn, side)
        vals = psi[planes].reshape(nf, nxy)
        out[planes] -= _sigma_apply_end(jn, md, vals).reshape(nf, jn.ny, jn.nx)
    return out


def apply_P(jn, alpha: float, gamma: np.ndarray) -> np.ndarray:
    """Eq. 10 with the six face neighbours, C_0 = 1, C_1 = exp(-alpha)."""
    c1 = np.exp(-alpha)
    g = np.asarray(gamma)
    out = g.copy()
    out = out + c1 * (np.roll(g, 1, axis=2) + np.roll(g, -1, axis=2))
    out = out + c1 * (np.roll(g, 1, axis=1) + np.roll(g, -1, axis=1))
    zp = np.zeros_like(g)
    zp[1:] = g[:-1]
    zm = np.zeros_like(g)
    zm[:-1] = g[1:]
    return out + c1 * (zp + zm)


def P_matrix(jn, alpha: float) -> sp.csr_matrix:
    """Eq. 10 as an explicit sparse matrix (six face neighbours)."""
    c1 = np.exp(-alpha)
    w1 = np.array([0.0, 1.0])   # nearest-neighbour adjacency
    Ix, Iy, Iz = sp.identity(jn.nx), sp.identity(jn.ny), sp.identity(jn.nz)
    Ax = _fd_matrix_periodic(jn.nx, w1)
    Ay = _fd_matrix_periodic(jn.ny, w1)
    Az = _fd_matrix_truncated(jn.nz, w1)
    adj = (sp.kron(sp.kron(Iz, Iy), Ax) + sp.kron(sp.kron(Iz, Ay), Ix)
           + sp.kron(sp.kron(Az, Iy), Ix))
    return (sp.identity(jn.npts) + c1 * adj).tocsr()


def free_inverse(jn, E: float, md: ModeData, r: np.ndarray) -> np.ndarray:
    """z = (E - T - H~)^{-1} r: the operator of Eqs. 7, 7-2 with V = 0 and no KB term,
    solved by sparse LU (r shaped [..., nz][ny][nx]; one factorisation for all)."""
    import scipy.sparse.linalg as spla
    flat = jn.copy_with(V=np.zeros_like(jn.V), projectors=[])
    lu = spla.splu(assemble_A_local(flat, E, md))
    r = np.asarray(r, dtype=np.complex128)
    vecs = r.reshape(-1, jn.npts)
    return np.stack([lu.solve(v) for v in vecs]).reshape(r.shape)
