"""The seeded synthetic junctions match the recipes the benchmark and the tests are
quoted on (grid, spacing, atoms, wells, projectors, electrodes, energy window, seed).

The paper's DFT potentials (Sec. III sodium wires, Sec. IV Ir/Au wires) are not
available; these junctions stand in for them, so their shapes are pinned here.
"""
import math

import numpy as np
import pytest

import iobm_synth as S


def check_projectors(jn, per_atom):
    assert len(jn.projectors) == per_atom * len(jn.atoms)
    dvol = jn.hx * jn.hy * jn.hz
    for p in jn.projectors:
        # normalised: h^3 sum p^2 = 1; sorted, distinct, inside the grid
        assert abs(dvol * float(np.dot(p.val, p.val)) - 1.0) < 1e-12
        assert np.all(np.diff(p.idx) > 0)
        assert p.idx.min() >= 0 and p.idx.max() < jn.npts
        # never on the N_f self-energy planes at either end
        k = p.idx // (jn.nx * jn.ny)
        assert k.min() >= jn.nf and k.max() < jn.nz - jn.nf


def check_wells(jn, depth, width):
    assert jn.V.shape == (jn.nz, jn.ny, jn.nx)
    assert np.all(jn.V <= 0.0)
    # the deepest point sits at an atom, within a grid step of it
    k, j, i = np.unravel_index(np.argmin(jn.V), jn.V.shape)
    r = np.array([i * jn.hx, j * jn.hy, k * jn.hz])
    dmin = min(np.linalg.norm(r - a) for a in jn.atoms)
    assert dmin <= math.sqrt(jn.hx ** 2 + jn.hy ** 2 + jn.hz ** 2)
    # one well's depth plus the overlap of its neighbours' tails
    assert depth * 0.8 <= -jn.V.min() <= depth * 1.5
    # flat (electrode) potential at the ends of the transition region
    assert np.max(np.abs(jn.V[0])) < 0.05 * depth and np.max(np.abs(jn.V[-1])) < 0.05 * depth


def test_wire48_bench_recipe():
    jn = S.wire48()
    assert (jn.nx, jn.ny, jn.nz, jn.nf) == (48, 48, 160, 4)
    assert jn.hx == jn.hy == jn.hz == 0.35
    assert jn.rs == 3.28 and len(jn.atoms) == 6 and jn.seed == 1000
    ef = S.fermi_energy(3.28)
    assert len(jn.energies) == 32
    assert abs(jn.energies[0] - (ef - 2.0 * S.EV)) < 1e-15
    assert abs(jn.energies[-1] - (ef + 0.5 * S.EV)) < 1e-15
    assert np.allclose(np.diff(jn.energies), (2.5 * S.EV) / 31, rtol=0, atol=1e-15)
    # a row along z, centred laterally; neighbours 6.8 bohr apart (jitter 0.1 per axis)
    a = jn.atoms
    assert np.all(np.abs(a[:, 0] - 0.5 * 48 * 0.35) <= 0.1)
    assert np.all(np.abs(a[:, 1] - 0.5 * 48 * 0.35) <= 0.1)
    assert np.all(np.abs(np.diff(a[:, 2]) - 6.8) <= 0.2)
    check_wells(jn, 0.5, 1.5)
    check_projectors(jn, 4)


def test_seeds_make_junctions_reproducible_and_distinct():
    a, b, c = S.wire48(0, n_energies=2), S.wire48(0, n_energies=2), S.wire48(1, n_energies=2)
    assert np.array_equal(a.V, b.V) and np.array_equal(a.atoms, b.atoms)
    assert [p.coupling for p in a.projectors] == [p.coupling for p in b.projectors]
    assert not np.array_equal(a.V, c.V)


def test_fermi_energy_free_electron_gas():
    # E_F = k_F^2 / 2 with k_F r_s = (9 pi / 4)^(1/3), i.e. 50.1 eV / (r_s / a_0)^2 —
    # the free-electron table value for sodium: r_s = 3.93 a_0, E_F = 3.24 eV
    assert abs(S.fermi_energy(3.93) * S.HARTREE_EV - 3.24) < 0.01
    for rs in (2.0, 3.28, 3.99):
        assert abs(S.fermi_energy(rs) * S.HARTREE_EV * rs * rs - 50.1) < 0.05
        kf = math.sqrt(2.0 * S.fermi_energy(rs))
        assert abs(kf * rs - (9.0 * math.pi / 4.0) ** (1.0 / 3.0)) < 1e-14


def test_wire12_copy_is_the_same_box():
    fine, coarse = S.wire48(), S.wire12_copy()
    assert (coarse.nx, coarse.ny, coarse.nz) == (12, 12, 40) and coarse.hx == 1.4
    assert abs(coarse.nx * coarse.hx - fine.nx * fine.hx) < 1e-12
    assert abs(coarse.nz * coarse.hz - fine.nz * fine.hz) < 1e-12
    # the same atoms relative to the box centre, the same couplings, at E_F
    cf = fine.atoms - [0, 0, 0.5 * (fine.nz - 1) * fine.hz]
    cc = coarse.atoms - [0, 0, 0.5 * (coarse.nz - 1) * coarse.hz]
    assert np.allclose(cf, cc, atol=1e-12)
    assert [p.coupling for p in coarse.projectors] == [p.coupling for p in fine.projectors]
    assert np.array_equal(coarse.energies, [fine.e_fermi])
    assert np.array_equal(S.wire48_at_fermi().energies, [fine.e_fermi])


def test_wire128_recipe():
    jn = S.wire128()
    assert (jn.nx, jn.ny, jn.nz) == (128, 128, 256) and jn.hx == 0.3
    assert jn.rs == 2.0 and len(jn.atoms) == 7 and len(jn.energies) == 8
    assert np.all(np.abs(np.diff(jn.atoms[:, 2]) - 4.3) <= 0.2)
    check_wells(jn, 2.0, 1.5)
    check_projectors(jn, 9)


@pytest.mark.parametrize("natom", [3, 5, 8])
def test_na_wire_geometry_of_sec_iii(natom):
    jn = S.na_wire(natom)
    d = 0.5 * math.sqrt(3.0) * 8.11   # Na [110] nearest-neighbour distance
    assert (jn.nx, jn.ny) == (36, 36) and abs(jn.nx * jn.hx - 25.66) < 1e-12
    assert jn.nz == 60 + 10 * (natom - 1)
    assert abs(jn.nz * jn.hz - ((natom - 1) * d + 42.12)) < 1e-12
    assert jn.rs == 3.99 and not jn.projectors
    assert np.array_equal(jn.energies, [S.fermi_energy(3.99)])
    assert len(jn.atoms) == natom
    assert np.all(np.abs(np.diff(jn.atoms[:, 2]) - d) <= 0.2)
    check_wells(jn, 0.3, 1.8)


def smooth_235(n):
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def test_batch_junctions_span_the_uneven_mix():
    sizes, nzs, natoms, rss = set(), [], [], []
    for j in range(48):
        jn = S.batch_junction(j, n_energies=2)
        assert jn.nx == jn.ny and smooth_235(jn.nx) and 24 <= jn.nx <= 64
        assert 96 <= jn.nz <= 256 and jn.hx == 0.35
        assert 2 <= len(jn.atoms) <= 8 and 2.0 <= jn.rs <= 4.0
        assert jn.energies[0] < jn.e_fermi < jn.energies[-1]
        sizes.add(jn.nx)
        nzs.append(jn.nz)
        natoms.append(len(jn.atoms))
        rss.append(jn.rs)
    # an uneven mix: many lateral sizes, lengths and atom counts
    assert len(sizes) >= 8
    assert max(nzs) - min(nzs) >= 100 and len(set(natoms)) >= 5
    assert max(rss) - min(rss) >= 1.5
