"""Seeded synthetic junctions for the IOBM transport solve.

This module only *generates inputs*: grids, local potentials, Kleinman-Bylander
projector tables, jellium Wigner-Seitz radii and energy lists.  It holds none of
the transport method's arithmetic (no finite-difference weights, no lateral
modes, no self-energies), so that the FP64 oracle (``oracle/``) and the CUDA
path (``paper_1009_5300_gb300``) can both draw the same junctions from it
without sharing any of the computation they are compared on.

Units are Hartree atomic units (energies in Ha, lengths in bohr).

The junction shapes stand in for the paper's DFT potentials (Sec. III and IV:
Na, Ir and Au single-row nanowires between jellium electrodes), which are not
available: a row of atoms along z, centred laterally in a periodic x-y cell,
each atom a spherical Gaussian well plus optional s/p/d Gaussian projectors.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

HARTREE_EV = 27.211386245988
EV = 1.0 / HARTREE_EV

# 2,3,5-smooth lateral sizes used by the uneven batched workload.
SMOOTH_LATERAL = (24, 25, 27, 30, 32, 36, 40, 45, 48, 50, 54, 60, 64)


def fermi_energy(rs: float) -> float:
    """Free-electron Fermi energy of jellium with Wigner-Seitz radius rs (Ha).

    k_F = (9 pi / 4)^(1/3) / rs and E_F = k_F^2 / 2, measured from the flat
    electrode potential (taken as the zero of energy).
    """
    return (9.0 * math.pi / 4.0) ** (2.0 / 3.0) / (2.0 * rs * rs)


@dataclasses.dataclass
class Projector:
    """One KB projector p(r) on the grid: linear indices and values."""
    idx: np.ndarray        # int32, linear index (z*ny + y)*nx + x
    val: np.ndarray        # float64, p(r) at those points; h^3 sum p^2 = 1
    coupling: float        # E_p in Ha
    atom: int              # atom the projector belongs to


@dataclasses.dataclass
class Junction:
    """A transition region of nz planes (planes 0..N_z+1), nx*ny lateral points."""
    name: str
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    nf: int
    V: np.ndarray                       # float64 [nz][ny][nx], Ha
    projectors: List[Projector]
    rs: float
    energies: np.ndarray                # float64, Ha
    atoms: np.ndarray                   # float64 [natom][3] positions (x,y,z), bohr
    seed: int = 0

    @property
    def npts(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def e_fermi(self) -> float:
        return fermi_energy(self.rs)

    def projector_csr(self):
        """(row_ptr int64, idx int32, val float64, coupling float64) CSR arrays."""
        counts = [len(p.idx) for p in self.projectors]
        row_ptr = np.zeros(len(counts) + 1, dtype=np.int64)
        if counts:
            row_ptr[1:] = np.cumsum(counts)
        idx = (np.concatenate([p.idx for p in self.projectors]).astype(np.int32)
               if counts else np.zeros(0, np.int32))
        val = (np.concatenate([p.val for p in self.projectors]).astype(np.float64)
               if counts else np.zeros(0, np.float64))
        coupling = np.array([p.coupling for p in self.projectors], dtype=np.float64)
        return row_ptr, idx, val, coupling

    def copy_with(self, **kw) -> "Junction":
        return dataclasses.replace(self, **kw)


def _coords(nx, ny, nz, hx, hy, hz):
    z = np.arange(nz) * hz
    y = np.arange(ny) * hy
    x = np.arange(nx) * hx
    return np.meshgrid(z, y, x, indexing="ij")


def _periodic_delta(d, L):
    """Minimum-image lateral displacement."""
    return d - L * np.round(d / L)


def gaussian_wells(nx, ny, nz, hx, hy, hz, atoms, depth, width) -> np.ndarray:
    """V(r) = -sum_a depth * exp(-|r - R_a|^2 / (2 width^2)), laterally periodic
    (summed over the nearest lateral images)."""
    Z, Y, X = _coords(nx, ny, nz, hx, hy, hz)
    Lx, Ly = nx * hx, ny * hy
    V = np.zeros((nz, ny, nx))
    depths = np.broadcast_to(np.asarray(depth, dtype=np.float64), (len(atoms),))
    for a, R in enumerate(atoms):
        dz2 = (Z - R[2]) ** 2
        for ix in (-1, 0, 1):
            dx2 = (X - R[0] - ix * Lx) ** 2
            for iy in (-1, 0, 1):
                dy2 = (Y - R[1] - iy * Ly) ** 2
                V -= depths[a] * np.exp(-(dx2 + dy2 + dz2) / (2.0 * width * width))
    return V


def _angular(kind: str, dx, dy, dz):
    r2 = dx * dx + dy * dy + dz * dz
    table = {
        "s": np.ones_like(dx),
        "px": dx, "py": dy, "pz": dz,
        "dxy": dx * dy, "dyz": dy * dz, "dzx": dz * dx,
        "dx2y2": dx * dx - dy * dy, "dz2": 3.0 * dz * dz - r2,
    }
    return table[kind]


SP = ("s", "px", "py", "pz")
SPD = SP + ("dxy", "dyz", "dzx", "dx2y2", "dz2")


def kb_projectors(nx, ny, nz, hx, hy, hz, atoms, kinds: Sequence[str], rng,
                  radius=3.0, radial_width=1.0, coupling_sigma=0.3) -> List[Projector]:
    """Gaussian-type KB projectors: angular(kind) * exp(-r^2/(2 w^2)) truncated at
    `radius`, normalised so that hx*hy*hz*sum p^2 = 1; coupling ~ N(0, sigma) Ha."""
    Lx, Ly = nx * hx, ny * hy
    dvol = hx * hy * hz
    out: List[Projector] = []
    for a, R in enumerate(atoms):
        # bounding box in index space (lateral indices wrap)
        kz0 = int(math.floor((R[2] - radius) / hz)) - 1
        kz1 = int(math.ceil((R[2] + radius) / hz)) + 1
        if kz0 < 0 or kz1 > nz - 1:
            raise ValueError("projector support leaves the transition region in z")
        ks = np.arange(kz0, kz1 + 1)
        jy = np.arange(int(math.floor((R[1] - radius) / hy)) - 1, int(math.ceil((R[1] + radius) / hy)) + 2)
        ix = np.arange(int(math.floor((R[0] - radius) / hx)) - 1, int(math.ceil((R[0] + radius) / hx)) + 2)
        # a box at least as wide as the cell covers every lateral point once
        if len(jy) >= ny:
            jy = np.arange(ny)
        if len(ix) >= nx:
            ix = np.arange(nx)
        KZ, JY, IX = np.meshgrid(ks, jy, ix, indexing="ij")
        dz = KZ * hz - R[2]
        dy = _periodic_delta(JY * hy - R[1], Ly)
        dx = _periodic_delta(IX * hx - R[0], Lx)
        r2 = dx * dx + dy * dy + dz * dz
        inside = r2 <= radius * radius
        lin = (KZ * ny + np.mod(JY, ny)) * nx + np.mod(IX, nx)
        lin = lin[inside]
        order = np.argsort(lin, kind="stable")
        lin = lin[order]
        if len(np.unique(lin)) != len(lin):
            raise ValueError("projector support wraps onto itself")
        g = np.exp(-r2[inside] / (2.0 * radial_width ** 2))[order]
        for kind in kinds:
            ang = _angular(kind, dx[inside][order], dy[inside][order], dz[inside][order])
            v = ang * g
            nrm = math.sqrt(dvol * float(np.dot(v, v)))
            v = v / nrm
            out.append(Projector(idx=lin.astype(np.int32), val=v.astype(np.float64),
                                 coupling=float(rng.normal(0.0, coupling_sigma)), atom=a))
    return out


def wire_atoms(nx, ny, nz, hx, hy, hz, natom, spacing, rng, jitter=0.1) -> np.ndarray:
    """A single-row wire along z, centred laterally and in z, with uniform
    +-jitter per coordinate."""
    Lx, Ly = nx * hx, ny * hy
    zc = 0.5 * (nz - 1) * hz
    zs = zc + (np.arange(natom) - 0.5 * (natom - 1)) * spacing
    atoms = np.stack([np.full(natom, 0.5 * Lx), np.full(natom, 0.5 * Ly), zs], axis=1)
    atoms = atoms + rng.uniform(-jitter, jitter, size=atoms.shape)
    return atoms


def make_wire(name, nx, ny, nz, h, natom, spacing, depth, width, rs, energies,
              kb_kinds: Optional[Sequence[str]], seed, nf=4, kb_radius=3.0,
              kb_width=1.0) -> Junction:
    rng = np.random.default_rng(seed)
    atoms = wire_atoms(nx, ny, nz, h, h, h, natom, spacing, rng)
    V = gaussian_wells(nx, ny, nz, h, h, h, atoms, depth, width)
    projs = (kb_projectors(nx, ny, nz, h, h, h, atoms, kb_kinds, rng, radius=kb_radius,
                           radial_width=kb_width) if kb_kinds else [])
    return Junction(name=name, nx=nx, ny=ny, nz=nz, hx=h, hy=h, hz=h, nf=nf, V=V,
                    projectors=projs, rs=rs, energies=np.asarray(energies, dtype=np.float64),
                    atoms=atoms, seed=seed)


# ---------------------------------------------------------------------------
# The five workloads.  Seeds are (workload index) * 1000 + junction id.

def wire16(junction_id: int = 0) -> Junction:
    """3-atom wire of Gaussian wells (0.5 Ha, width 1.5, spacing 6.8) on a
    16x16x64 grid, h=0.4, r_s=3.28 jellium, one energy at E_F, 9-point FD."""
    rs = 3.28
    return make_wire("wire16", 16, 16, 64, 0.4, 3, 6.8, 0.5, 1.5, rs,
                     [fermi_energy(rs)], None, seed=0 * 1000 + junction_id)


def wire48(junction_id: int = 0, n_energies: int = 32) -> Junction:
    """6-atom wire on a 48x48x160 grid, h=0.35, r_s=3.28, Gaussian wells plus
    s/p KB projectors; energies uniform in [E_F - 2 eV, E_F + 0.5 eV]."""
    rs = 3.28
    ef = fermi_energy(rs)
    E = np.linspace(ef - 2.0 * EV, ef + 0.5 * EV, n_energies)
    return make_wire("wire48", 48, 48, 160, 0.35, 6, 6.8, 0.5, 1.5, rs, E, SP,
                     seed=1 * 1000 + junction_id)


def batch_junction(junction_id: int, n_energies: int = 16) -> Junction:
    """One junction of the uneven batched workload: lateral N from a 2,3,5-smooth
    set in [24, 64], N_z in [96, 256], h=0.35, 2-8 atoms, r_s in [2, 4]."""
    rng = np.random.default_rng(2 * 1000 + junction_id)
    n = int(rng.choice(SMOOTH_LATERAL))
    nz = int(rng.integers(96, 257))
    natom = int(rng.integers(2, 9))
    rs = float(rng.uniform(2.0, 4.0))
    h = 0.35
    Lz = (nz - 1) * h
    spacing = min(6.8, (Lz - 8.0) / max(natom - 1, 1))
    ef = fermi_energy(rs)
    E = np.linspace(ef - 1.0 * EV, ef + 0.5 * EV, n_energies)
    seed = int(rng.integers(0, 2 ** 31 - 1))
    return make_wire(f"batch{junction_id}", n, n, nz, h, natom, spacing, 0.5, 1.5, rs, E, None,
                     seed=seed)


def wire48_at_fermi(junction_id: int = 0) -> Junction:
    """The 48x48x160 wire at E_F only (gradient workload)."""
    j = wire48(junction_id)
    return j.copy_with(name="wire48_ef", energies=np.array([j.e_fermi]))


def wire12_copy(junction_id: int = 0) -> Junction:
    """The same physical box as the 48x48x160 wire (16.8 x 16.8 x 56 bohr) on a
    12x12x40 grid (h = 1.4 bohr), same atoms, wells and projector shapes, at E_F."""
    fine = wire48(junction_id)
    h = 1.4
    nx = ny = 12
    nz = 40
    # the fine grid's plane 0 and plane 159 are at z=0 and 159*0.35; keep the
    # physical atom positions relative to the box centre
    shift = 0.5 * (nz - 1) * h - 0.5 * (fine.nz - 1) * fine.hz
    atoms = fine.atoms.copy()
    atoms[:, 2] += shift
    V = gaussian_wells(nx, ny, nz, h, h, h, atoms, 0.5, 1.5)
    rng = np.random.default_rng(3 * 1000 + junction_id)
    projs = kb_projectors(nx, ny, nz, h, h, h, atoms, SP, rng)
    # reuse the fine junction's couplings so the copy is the same physical model
    for p_c, p_f in zip(projs, fine.projectors):
        p_c.coupling = p_f.coupling
    return Junction(name="wire12", nx=nx, ny=ny, nz=nz, hx=h, hy=h, hz=h, nf=4, V=V,
                    projectors=projs, rs=fine.rs, energies=np.array([fine.e_fermi]),
                    atoms=atoms, seed=3 * 1000 + junction_id)


def wire128(junction_id: int = 0, n_energies: int = 8) -> Junction:
    """Large cross-section: 128x128x256, h=0.3, r_s=2.0, 7 atoms at 4.3 bohr,
    deep wells (2.0 Ha) plus s/p/d-like KB projectors, 8 energies."""
    rs = 2.0
    ef = fermi_energy(rs)
    E = np.linspace(ef - 1.0 * EV, ef + 0.5 * EV, n_energies)
    return make_wire("wire128", 128, 128, 256, 0.3, 7, 4.3, 2.0, 1.5, rs, E, SPD,
                     seed=4 * 1000 + junction_id)


def na_wire(natom: int, junction_id: int = 0, nxy: int = 36) -> Junction:
    """Synthetic stand-in for the Sec. III sodium wires (the paper's DFT potentials are
    not reproduced): a single row of natom Gaussian wells (0.3 Ha, width 1.8 bohr) at
    the Na [110] spacing d = (sqrt(3)/2) 8.11 bohr between r_s = 3.99 jellium
    electrodes; lateral cell 25.66 bohr on nxy x nxy points (36 in Sec. III),
    N_z = 60 + 10 (natom - 1) planes over L_z = (natom - 1) d + 42.12 bohr; at E_F."""
    rs = 3.99
    d = 0.5 * np.sqrt(3.0) * 8.11
    L = 25.66
    nz = 60 + 10 * (natom - 1)
    hz = ((natom - 1) * d + 42.12) / nz
    h = L / nxy
    rng = np.random.default_rng(5 * 1000 + 10 * natom + junction_id)
    atoms = wire_atoms(nxy, nxy, nz, h, h, hz, natom, d, rng)
    V = gaussian_wells(nxy, nxy, nz, h, h, hz, atoms, 0.3, 1.8)
    return Junction(name=f"na{natom}", nx=nxy, ny=nxy, nz=nz, hx=h, hy=h, hz=hz, nf=4, V=V,
                    projectors=[], rs=rs, energies=np.array([fermi_energy(rs)]), atoms=atoms,
                    seed=5 * 1000 + 10 * natom + junction_id)


def small_wire(nx=8, ny=8, nz=24, h=0.5, natom=2, spacing=3.0, depth=0.5, width=1.0,
               rs=3.28, energies=None, kb_kinds=None, seed=12345, nf=4, kb_radius=1.5,
               kb_width=0.6) -> Junction:
    """Tiny junctions for tests (sizes the direct oracle finishes in seconds)."""
    ef = fermi_energy(rs)
    if energies is None:
        energies = [ef]
    return make_wire(f"small{nx}x{ny}x{nz}", nx, ny, nz, h, natom, spacing, depth, width, rs,
                     energies, kb_kinds, seed=seed, nf=nf, kb_radius=kb_radius,
                     kb_width=kb_width)


def random_field(shape, seed, dtype=np.complex128) -> np.ndarray:
    """Seeded complex Gaussian test vector."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return a.astype(dtype)


WORKLOADS = {
    "wire16": wire16,
    "wire48": wire48,
    "batch": batch_junction,
    "wire48_ef": wire48_at_fermi,
    "wire12": wire12_copy,
    "wire128": wire128,
}
