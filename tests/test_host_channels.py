"""The library's host-side channel set-up against the oracle (no GPU needed).

Two independent routes: the library finds the Bloch roots through the
Chebyshev reduction in u = (lambda + 1/lambda)/2 and its own root finder; the
oracle hands the degree-2N_f polynomial to numpy.roots."""
import numpy as np
import pytest

import iobm_synth as S
from oracle import modes


@pytest.fixture(scope="module")
def host():
    from paper_1009_5300_gb300 import build_library
    build_library()
    from paper_1009_5300_gb300.solver import channels_host
    return channels_host


CASES = [(16, 16, 0.4, 0.4, 0.4, 4, S.fermi_energy(3.28)),
         (48, 48, 0.35, 0.35, 0.35, 4, S.fermi_energy(3.28)),
         (12, 10, 0.5, 0.45, 0.4, 1, 0.9),
         (25, 27, 0.35, 0.35, 0.35, 4, 0.3),
         (46, 46, 15.07 / 46, 15.07 / 46, 15.07 / 46, 4, S.fermi_energy(1.36))]


@pytest.mark.parametrize("nx,ny,hx,hy,hz,nf,E", CASES)
def test_channels_match_oracle(host, nx, ny, hx, hy, hz, nf, E):
    check_against_oracle(host, nx, ny, hx, hy, hz, nf, E, (0.0, 0.0))


# lateral Bloch vectors as fractions of pi / L per axis
@pytest.mark.parametrize("case,fx,fy", [(0, 0.31, -0.57), (2, -0.8, 0.45), (3, 0.5, 0.0)])
def test_channels_match_oracle_at_kappa(host, case, fx, fy):
    nx, ny, hx, hy, hz, nf, E = CASES[case]
    kappa = (fx * np.pi / (nx * hx), fy * np.pi / (ny * hy))
    check_against_oracle(host, nx, ny, hx, hy, hz, nf, E, kappa)


def check_against_oracle(host, nx, ny, hx, hy, hz, nf, E, kappa):
    lib = host(nx, ny, hx, hy, hz, nf, E, want_sigma=True, kappa=kappa)
    md = modes.mode_data(nx, ny, hx, hy, hz, nf, E, kappa=kappa)
    opens = md.open_modes
    assert lib["n_open"] == len(opens)
    assert np.array_equal(lib["nu"], md.nu[opens])
    assert np.allclose(lib["vel"], md.vel[opens], rtol=1e-11, atol=0)
    lam_or = md.lam[opens, md.prop[opens]]
    assert np.max(np.abs(lib["lam"] - lam_or)) < 1e-11
    for c, m in enumerate(opens):
        bo = modes.incident_source_mode(md, m)
        assert np.max(np.abs(lib["btilde"][c] - bo)) < 1e-10 * np.max(np.abs(bo))
        # mrow: t = mrow . psi~ must return the coefficient of the propagating root
        d = np.arange(nf)
        Qin = md.lam[m][None, :] ** (-d[:, None])
        row = np.linalg.inv(Qin)[md.prop[m]]
        assert np.max(np.abs(lib["mrow"][c] - row)) < 1e-9 * np.max(np.abs(row))
    sig = lib["sigma"]
    for m in range(len(md.nu)):
        kx = md.nu[m, 0] % nx
        ky = md.nu[m, 1] % ny
        ref = md.sigma[m]
        assert np.max(np.abs(sig[ky, kx] - ref)) < 1e-10 * np.max(np.abs(ref))


def test_threshold_reported(host):
    from paper_1009_5300_gb300._lib import IOBMError, IOBM_E_THRESHOLD
    md = modes.mode_data(8, 8, 0.4, 0.4, 0.4, 4, 0.3)
    e_perp = np.unique(np.round(md.eps_perp, 12))
    with pytest.raises(IOBMError) as ei:
        host(8, 8, 0.4, 0.4, 0.4, 4, float(e_perp[1]) + 1e-12)
    assert ei.value.code == IOBM_E_THRESHOLD


def test_ir_au_channel_count(host):
    # Sec. IV: 37 incident waves for the Ir and Au electrodes
    for rs, L, N in ((1.36, 15.07, 46), (1.35, 15.38, 48)):
        h = L / N
        assert host(N, N, h, h, h, 4, S.fermi_energy(rs))["n_open"] == 37
