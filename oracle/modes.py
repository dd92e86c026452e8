"""Electrode channels, generalised Bloch roots and the per-mode self-energy.

Paper passages followed:

* Lateral modes: G_nu = 2 pi nu / L with nu = -N/2 .. N/2-1 (Eq. 8 and the
  Appendix), and the lateral Fourier transform with the 1/N_xy on the forward
  side (Eq. 19).  The lateral Bloch vector kappa of Eq. 8 shifts every mode to
  G_nu + kappa (the wave picks up exp(i kappa L) across a lateral period); it is
  a parameter here, zero by default (the examples of Sec. III).
* The electrode recurrence: in a flat (zero-potential) jellium electrode
  Eq. 2 decouples per lateral mode nu into the 1D recurrence

      (E - eps_perp(nu)) psi_k + (1/(2 h_z^2)) sum_{n=-N_f}^{N_f} w_|n| psi_{k+n} = 0,

  whose solutions psi_k = lambda^k are the generalised Bloch states of
  Eqs. 6 and 17.  For N_f = 1 the characteristic equation is
  lambda^2 + 2 chi lambda + 1 = 0 with chi of Eq. 9, i.e. the root pair
  omega_1 omega_2 = 1 of Eq. A-08, and lambda = exp(i k_z h_z) with k_z of
  Eq. 8.5.  For general N_f it is the degree-2N_f polynomial obtained by
  multiplying the recurrence symbol by lambda^N_f; this oracle hands it to
  numpy.roots.
* Right-going (transmitted, Eq. 6) roots: |lambda| < 1, or |lambda| = 1 with a
  positive group velocity v = (1/h_z) sum_n n w_n sin(n k h_z).  For N_f = 1 this
  is the branch rule stated after Eq. 9 (k_z > 0, or -i k_z > 0).
* Self-energy per mode (Eqs. 17-1/17-2 written in the lateral Fourier basis,
  where Q^A is diagonal in nu): with depth index d = 0 .. N_f-1 counted inward
  from the outermost transition plane and e = 1 .. N_f counted outward into the
  electrode,

      Q_in[d, j]  = lambda_j^(-d),    Q_out[e-1, j] = lambda_j^(e),
      K[d, e-1]   = w_{d+e} / (2 h_z^2)   (zero when d + e > N_f),
      Sigma~_nu   = -K Q_out Q_in^{-1}.

  For N_f = 1 this is -(1/(2 h_z^2)) exp(i k_z h_z), Eq. 18-2.  The left and
  right electrodes have the same Sigma~ in depth coordinates (the jellium
  electrodes are identical, Sec. II).
* Incident source (Eq. 7, generalised to N_f planes): for an incident wave
  lambda_in^k on the entry side, the source on the first N_f transition rows is
  b~[d] = -sum_e K[d,e] lambda_in^(-e) - sum_d' Sigma~[d,d'] lambda_in^(d').
  For N_f = 1 this is B^dagger Phi_in(z_-1) - Sigma Phi_in(z_0).

Readings where the paper is silent (listed with the others in the design notes):
channels within 1e-9 Ha of a lateral threshold or of the band top are
rejected; a root counts as unit-modulus when ||lambda| - 1| < 1e-10.

Pinned by: Eq. 18-2 / A-10 for N_f = 1 (closed form); the surface Green's
function of a long explicit chain at complex energy for N_f = 4 (brute force,
Eq. A-01); channel counts printed for the Ir/Au cells (Sec. IV);
tests/test_oracle_modes.py.
"""
from __future__ import annotations

import dataclasses
from typing import List, Tuple

import numpy as np

from .fd import second_derivative_weights

UNIT_TOL = 1e-10
THRESHOLD_TOL = 1e-9


class ThresholdError(ValueError):
    """Energy too close to a channel threshold (zero group velocity)."""


def lateral_indices(n: int) -> np.ndarray:
    """nu = -N/2 .. N/2-1 (for odd N: -(N-1)/2 .. (N-1)/2)."""
    return np.arange(-(n // 2), n - n // 2)


def lateral_G(n: int, h: float) -> np.ndarray:
    return 2.0 * np.pi * lateral_indices(n) / (n * h)


def lateral_energy_1d(G: np.ndarray, h: float, w: np.ndarray) -> np.ndarray:
    """-1/2 times the FD second-derivative symbol along one lateral axis."""
    s = w[0] + 2.0 * sum(w[n] * np.cos(n * G * h) for n in range(1, len(w)))
    return -0.5 * s / (h * h)


def band_top_z(hz: float, w: np.ndarray) -> float:
    """1D kinetic energy at k h_z = pi (top of the electrode z band)."""
    s = w[0] + 2.0 * sum(w[n] * (-1.0) ** n for n in range(1, len(w)))
    return -0.5 * s / (hz * hz)


@dataclasses.dataclass
class ModeData:
    """Per-energy electrode data for every lateral mode (flattened nu_y-major)."""
    E: float
    nf: int
    hz: float
    w: np.ndarray                 # FD weights
    nu: np.ndarray                # [Nmodes, 2] (nu_x, nu_y)
    eps_perp: np.ndarray          # [Nmodes]
    lam: np.ndarray               # [Nmodes, nf] right-going roots
    prop: np.ndarray              # [Nmodes] index of the propagating root or -1
    vel: np.ndarray               # [Nmodes] group velocity of propagating root (0 if closed)
    sigma: np.ndarray             # [Nmodes, nf, nf] Sigma~ in depth coordinates
    K: np.ndarray                 # [nf, nf] coupling to the electrode planes
    kappa: Tuple[float, float] = (0.0, 0.0)   # lateral Bloch vector (Eq. 8)

    @property
    def open_modes(self) -> np.ndarray:
        return np.nonzero(self.prop >= 0)[0]


def velocity(lam: complex, w: np.ndarray, hz: float) -> float:
    kh = np.angle(lam)
    return float(sum(n * w[n] * np.sin(n * kh) for n in range(1, len(w))) / hz)


def z_roots(E_minus_eps: float, w: np.ndarray, hz: float) -> np.ndarray:
    """All 2 N_f roots of lambda^N_f [2 h_z^2 (E - eps) + w_0 + sum w_n (lambda^n + lambda^-n)]."""
    nf = len(w) - 1
    coeffs = np.zeros(2 * nf + 1, dtype=np.result_type(float, E_minus_eps))
    # numpy.roots: highest degree first; power p -> position 2nf - p
    for n in range(1, nf + 1):
        coeffs[2 * nf - (nf + n)] = w[n]
        coeffs[2 * nf - (nf - n)] = w[n]
    coeffs[2 * nf - nf] = w[0] + 2.0 * hz * hz * E_minus_eps
    roots = np.roots(coeffs)
    # two Newton steps on the same polynomial to polish the companion eigenvalues
    dcoeffs = np.polyder(coeffs)
    for _ in range(2):
        roots = roots - np.polyval(coeffs, roots) / np.polyval(dcoeffs, roots)
    return roots


def right_going(roots: np.ndarray, w: np.ndarray, hz: float) -> Tuple[np.ndarray, int, float]:
    """Select the N_f right-going roots; return (roots, index of propagating, velocity)."""
    nf = len(w) - 1
    sel = []
    prop = -1
    vprop = 0.0
    for lam in roots:
        a = abs(lam)
        if a < 1.0 - UNIT_TOL:
            sel.append(lam)
        elif abs(a - 1.0) <= UNIT_TOL:
            v = velocity(lam, w, hz)
            if v > 0.0:
                prop = len(sel)
                vprop = v
                sel.append(lam / a)
    if len(sel) != nf:
        raise ThresholdError(f"found {len(sel)} right-going roots, expected {nf}")
    return np.array(sel), prop, vprop


def coupling_matrix(w: np.ndarray, hz: float) -> np.ndarray:
    nf = len(w) - 1
    K = np.zeros((nf, nf))
    for d in range(nf):
        for e in range(1, nf + 1):
            if d + e <= nf:
                K[d, e - 1] = w[d + e] / (2.0 * hz * hz)
    return K


def sigma_mode(lam: np.ndarray, K: np.ndarray) -> np.ndarray:
    """Sigma~ = -K Q_out Q_in^{-1} (Eqs. 17-1/17-2 in one lateral mode)."""
    nf = len(lam)
    d = np.arange(nf)
    Qin = lam[None, :] ** (-d[:, None])
    Qout = lam[None, :] ** (d[:, None] + 1)
    return -K @ Qout @ np.linalg.inv(Qin)


def mode_data(nx: int, ny: int, hx: float, hy: float, hz: float, nf: int, E: float,
              check_threshold: bool = True, kappa=(0.0, 0.0)) -> ModeData:
    w = second_derivative_weights(nf)
    kappa = (float(kappa[0]), float(kappa[1]))
    Gx = lateral_G(nx, hx) + kappa[0]     # G_nu + kappa (Eq. 8)
    Gy = lateral_G(ny, hy) + kappa[1]
    ex = lateral_energy_1d(Gx, hx, w)
    ey = lateral_energy_1d(Gy, hy, w)
    nux, nuy = lateral_indices(nx), lateral_indices(ny)
    K = coupling_matrix(w, hz)
    top = band_top_z(hz, w)
    nmodes = nx * ny
    nu = np.zeros((nmodes, 2), dtype=np.int64)
    eps = np.zeros(nmodes)
    lam = np.zeros((nmodes, nf), dtype=np.complex128)
    prop = np.full(nmodes, -1, dtype=np.int64)
    vel = np.zeros(nmodes)
    sigma = np.zeros((nmodes, nf, nf), dtype=np.complex128)
    m = 0
    for iy in range(ny):
        for ix in range(nx):
            e_perp = ex[ix] + ey[iy]
            if check_threshold and (abs(E - e_perp) < THRESHOLD_TOL
                                    or abs(E - e_perp - top) < THRESHOLD_TOL):
                raise ThresholdError(f"E={E} within {THRESHOLD_TOL} Ha of a threshold of mode "
                                     f"({nux[ix]},{nuy[iy]})")
            roots = z_roots(E - e_perp, w, hz)
            sel, p, v = right_going(roots, w, hz)
            nu[m] = (nux[ix], nuy[iy])
            eps[m] = e_perp
            lam[m] = sel
            prop[m] = p
            vel[m] = v
            sigma[m] = sigma_mode(sel, K)
            m += 1
    return ModeData(E=E, nf=nf, hz=hz, w=w, nu=nu, eps_perp=eps, lam=lam, prop=prop,
                    vel=vel, sigma=sigma, K=K, kappa=kappa)


def incident_source_mode(md: ModeData, m: int) -> np.ndarray:
    """b~[d] for a unit incident wave lambda_in^k in mode m (Eq. 7 for N_f planes)."""
    lam_in = md.lam[m, md.prop[m]]
    nf = md.nf
    e = np.arange(1, nf + 1)
    d = np.arange(nf)
    return -md.K @ (lam_in ** (-e)) - md.sigma[m] @ (lam_in ** d)


def count_open_channels(nx, ny, hx, hy, hz, nf, E, kappa=(0.0, 0.0)) -> int:
    """Number of propagating right-going channels at energy E."""
    md = mode_data(nx, ny, hx, hy, hz, nf, E, check_threshold=False, kappa=kappa)
    return int(np.sum(md.prop >= 0))


def lateral_phase(nx: int, ny: int, hx: float, hy: float, md: ModeData) -> np.ndarray:
    """F[m, l] = exp(-i (G_m + kappa) . r_l) for all modes m and lateral points l = y*nx + x."""
    x = np.arange(nx) * hx
    y = np.arange(ny) * hy
    Gx = 2.0 * np.pi * md.nu[:, 0] / (nx * hx) + md.kappa[0]
    Gy = 2.0 * np.pi * md.nu[:, 1] / (ny * hy) + md.kappa[1]
    ph = np.exp(-1j * (Gy[:, None, None] * y[None, :, None] + Gx[:, None, None] * x[None, None, :]))
    return ph.reshape(len(md.nu), nx * ny)


def eq19_forward(nx, ny, hx, hy, md: ModeData, plane: np.ndarray) -> np.ndarray:
    """psi~_nu = (1/N_xy) sum_l exp(-i (G_nu + kappa) . r_l) psi(r_l)  (Eq. 19), as an
    explicit sum."""
    F = lateral_phase(nx, ny, hx, hy, md)
    return F @ plane.reshape(-1) / (nx * ny)


def mode_order(md: ModeData) -> List[Tuple[int, int]]:
    return [tuple(int(a) for a in md.nu[m]) for m in range(len(md.nu))]
