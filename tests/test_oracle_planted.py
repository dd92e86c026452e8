"""The oracle's pins catch plausible mistakes: each test plants one slip in the oracle
(a patched copy of one of its functions, on the CPU) and checks that at least one pin
then fails — the symmetry pins of test_oracle_symmetries, or the central-difference
gradient at a generic Bloch vector of test_oracle_bloch (at kappa = pi / L_x, the
supercell's second fold, A(kappa) is complex symmetric, so a missing transposition of
the adjoint solve shows only at a generic kappa).  The slips are the kind an implementation of
Eqs. 8, 19 and the N_f end planes of Eq. 7 can make: a transposed lateral operand, a
dropped Bloch vector in the modes, the phases or the wrapped couplings, an end plane
taken in the wrong order or one plane in, a projected amplitude with the right modulus
and the wrong phase (which current conservation cannot see), an adjoint solve that
treats A(kappa) as complex symmetric, a wrong power or axis of the grid spacing."""
import numpy as np
import pytest

import oracle.modes as M
import oracle.operator as O
import oracle.transport as T
import test_oracle_bloch as TB
import test_oracle_symmetries as TS

PINS = [("supercell", TS.test_supercell_folds_two_bloch_vectors, ()),
        ("transpose", TS.test_transposed_cell_same_conductance, ()),
        ("translate", TS.test_lateral_translation_same_t_and_r, (1, 3)),
        ("mirror", TS.test_mirror_image_swaps_the_electrodes, (4,)),
        ("unitarity", TS.test_scattering_matrix_unitary, (4, (0.0, 0.0))),
        ("supercell gradient", TS.test_supercell_gradient_folds_two_bloch_vectors, ()),
        ("gradient at kappa", TB.test_gradient_at_kappa_matches_finite_differences, ()),
        ("scaling", TS.test_dimensional_scaling, (4,)),
        ("flat anisotropic", TS.test_flat_potential_anisotropic_grid, (4,))]

_mode_data = M.mode_data


def _phase(nx, ny, hx, hy, md, Gx, Gy):
    x = np.arange(nx) * hx
    y = np.arange(ny) * hy
    ph = np.exp(-1j * (Gy[:, None, None] * y[None, :, None] + Gx[:, None, None] * x[None, None, :]))
    return ph.reshape(len(md.nu), nx * ny)


def phase_gy_from_x(nx, ny, hx, hy, md):
    Gx = 2 * np.pi * md.nu[:, 0] / (nx * hx) + md.kappa[0]
    Gy = 2 * np.pi * md.nu[:, 1] / (nx * hx) + md.kappa[1]     # slip: n_x h_x for y
    return _phase(nx, ny, hx, hy, md, Gx, Gy)


def phase_without_kappa(nx, ny, hx, hy, md):
    Gx = 2 * np.pi * md.nu[:, 0] / (nx * hx)                    # slip: kappa dropped
    Gy = 2 * np.pi * md.nu[:, 1] / (ny * hy)
    return _phase(nx, ny, hx, hy, md, Gx, Gy)


def modes_hy_from_hx(nx, ny, hx, hy, hz, nf, E, check_threshold=True, kappa=(0.0, 0.0)):
    return _mode_data(nx, ny, hx, hx, hz, nf, E, check_threshold, kappa)   # slip: h_y <- h_x


def modes_without_kappa(nx, ny, hx, hy, hz, nf, E, check_threshold=True, kappa=(0.0, 0.0)):
    md = _mode_data(nx, ny, hx, hy, hz, nf, E, check_threshold, (0.0, 0.0))  # slip: eps(G)
    md.kappa = (float(kappa[0]), float(kappa[1]))
    return md


def wrap_without_phase(jn, kappa):
    return None, None                                            # slip: plain periodic wrap


def right_planes_in_depth_order(jn, side):
    # slip: the right electrode's planes taken from the interior outwards
    return np.arange(jn.nf) + (jn.nz - jn.nf) if side == "R" else np.arange(jn.nf)


def right_planes_one_in(jn, side):
    return jn.nz - 2 - np.arange(jn.nf) if side == "R" else np.arange(jn.nf)   # slip: shifted


_project = T.project


def project_conj_r(jn, md, psi, m_in, side):
    t, r = _project(jn, md, psi, m_in, side)
    return t, np.conj(r)                                         # slip: |r| right, phase wrong


def project_conj_t(jn, md, psi, m_in, side):
    t, r = _project(jn, md, psi, m_in, side)
    return np.conj(t), r                                         # slip: |t| right, phase wrong


def grad_adjoint_untransposed(jn, E, sol=None, kappa=(0.0, 0.0)):
    # slip: the adjoint waves solved with A instead of A^T, although A(kappa) is not
    # complex symmetric at kappa != 0
    import scipy.sparse.linalg as spla
    if sol is None:
        sol = T.solve(jn, E, kappa=kappa)
    md = sol.md
    lu = spla.splu(T.assemble_augmented(jn, E, md))
    nproj = len(jn.projectors)
    g = np.zeros((jn.nz, jn.ny, jn.nx))
    for o, m_out in enumerate(sol.open_modes):
        wv = T.exit_functional(jn, md, m_out, sol.side).reshape(-1)
        lam = lu.solve(np.concatenate([wv, np.zeros(nproj, np.complex128)]))[: jn.npts]
        lam = lam.reshape(jn.nz, jn.ny, jn.nx)
        for i in range(sol.psi.shape[0]):
            g += np.real(2.0 * sol.vel[o] / sol.vel[i] * np.conj(sol.t[o, i]) * lam * sol.psi[i])
    return g


_kb_factors = O.kb_factors
_coupling_matrix = M.coupling_matrix


def kb_volume_without_hz(jn):
    P, coupling, dvol = _kb_factors(jn)
    return P, coupling, jn.hx * jn.hy                            # slip: h_z dropped


def coupling_one_power_of_hz(w, hz):
    return _coupling_matrix(w, hz) * hz                          # slip: w / (2 h_z)


def modes_hz_from_hx(nx, ny, hx, hy, hz, nf, E, check_threshold=True, kappa=(0.0, 0.0)):
    return _mode_data(nx, ny, hx, hy, hx, nf, E, check_threshold, kappa)   # slip: h_z <- h_x


PLANTS = {
    "lateral phase G_y from n_x h_x": [(M, "lateral_phase", phase_gy_from_x),
                                       (O, "lateral_phase", phase_gy_from_x),
                                       (T, "lateral_phase", phase_gy_from_x)],
    "lateral phase without kappa": [(M, "lateral_phase", phase_without_kappa),
                                    (O, "lateral_phase", phase_without_kappa),
                                    (T, "lateral_phase", phase_without_kappa)],
    "mode tables with h_y = h_x": [(M, "mode_data", modes_hy_from_hx),
                                   (T, "mode_data", modes_hy_from_hx)],
    "mode energies without kappa": [(M, "mode_data", modes_without_kappa),
                                    (T, "mode_data", modes_without_kappa)],
    "wrapped couplings without phase": [(O, "_bloch_phases", wrap_without_phase)],
    "right end planes in depth order": [(O, "end_planes", right_planes_in_depth_order),
                                        (T, "end_planes", right_planes_in_depth_order)],
    "right end planes one plane in": [(O, "end_planes", right_planes_one_in),
                                      (T, "end_planes", right_planes_one_in)],
    "reflection amplitudes conjugated": [(T, "project", project_conj_r)],
    "transmission amplitudes conjugated": [(T, "project", project_conj_t)],
    "adjoint solve untransposed at kappa": [(T, "grad_V", grad_adjoint_untransposed)],
    "KB volume element without h_z": [(O, "kb_factors", kb_volume_without_hz),
                                      (T, "kb_factors", kb_volume_without_hz)],
    "self-energy coupling over h_z": [(M, "coupling_matrix", coupling_one_power_of_hz)],
    "electrode modes with h_x for h_z": [(M, "mode_data", modes_hz_from_hx),
                                         (T, "mode_data", modes_hz_from_hx)],
}


@pytest.mark.parametrize("plant", list(PLANTS))
def test_planted_slip_fails_a_symmetry_pin(plant, monkeypatch):
    for mod, attr, fn in PLANTS[plant]:
        monkeypatch.setattr(mod, attr, fn)
    failed = []
    for name, pin, args in PINS:
        try:
            pin(*args)
        except AssertionError:
            failed.append(name)
            break   # one failing pin shows the slip
    assert failed, f"'{plant}' passes every pin"
