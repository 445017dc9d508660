"""Seeded synthetic instances for the plane-wave multiple-scattering path.

This module only draws and lays out inputs: lattice vectors, plane-wave cutoff,
slice edges along the transport axis z, Gaussian wells, lead descriptions, and
the (E, k_par) points.  It holds none of the method's arithmetic (no G-vectors,
no Fourier coefficients, no matrices), so the CPU oracle and the CUDA path can
both consume it without sharing any of the computation.

Units are Rydberg atomic units (hbar^2/2m = 1, lengths in bohr, energies in
Ry), as in the paper's computational details (Sec. II B).

Geometry of the graphene-like side-contact junction (Sec. II B, Fig. 1):
the two sheets lie in the x-z plane, x is the periodic transverse direction
(a_x = 2.46 A), y is the vacuum direction (L_y = 20 A), z is the transport
direction.  The bottom sheet fills z in [0, 6 cells) and continues into the
left electrode; the top sheet fills z in [2, 8 cells) and continues into the
right electrode, so the sheets overlap over 4 of the 8 rectangular cells.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ANGSTROM = 1.8897261246  # bohr per angstrom
RYDBERG_EV = 13.605693   # eV per Ry

SEED_BASE = 1504_01462


@dataclasses.dataclass
class Lead:
    """A z-invariant electrode whose potential is the z-average of a periodic
    array of Gaussian wells (one period of length ``period`` along z).

    ``wells_xy`` are the transverse positions of the wells in one period.
    An empty lead (no wells) is the constant V = 0 electrode."""

    wells_xy: np.ndarray            # (n, 2)
    v0: np.ndarray                  # (n,)
    sigma: np.ndarray               # (n,)
    period: float = 1.0

    @staticmethod
    def free() -> "Lead":
        return Lead(np.zeros((0, 2)), np.zeros(0), np.zeros(0), 1.0)


@dataclasses.dataclass
class Instance:
    """One transport problem: cell, basis cutoff, slicing, wells, leads and
    the list of (E, k_par) points to evaluate."""

    a1: np.ndarray                  # (2,) transverse lattice vector, bohr
    a2: np.ndarray                  # (2,)
    ecut: float                     # |G|^2 <= ecut (Ry) for full shells
    ng_exact: int                   # >0: first ng_exact G by (|G|^2, m, n)
    z_edges: np.ndarray             # (n_slices+1,) increasing, bohr
    wells_xyz: np.ndarray           # (n_wells, 3): x, y transverse; z along transport
    v0: np.ndarray                  # (n_wells,) well depths, Ry (V = -v0 exp(..))
    sigma: np.ndarray               # (n_wells,) bohr
    lead_left: Lead
    lead_right: Lead
    energies: np.ndarray            # (npts,) Ry
    kpar: np.ndarray                # (npts, 2) 1/bohr
    slice_vg: np.ndarray | None = None   # optional explicit V^p(dG) tables (see below)
    lead_vg: tuple | None = None         # optional explicit lead tables
    vg_half: tuple = (0, 0)              # (Dm, Dn): table index ranges [-Dm,Dm]x[-Dn,Dn]
    name: str = ""
    # transverse displacement of each device well and of each electrode per
    # unit sheet gap (bohr/bohr); None when the instance has no gap parameter
    gap_rate_wells: np.ndarray | None = None   # (n_wells, 2)
    gap_rate_leads: np.ndarray | None = None   # (2, 2): left, right

    @property
    def n_slices(self) -> int:
        return len(self.z_edges) - 1


def _rng(cfg: int) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + cfg)


# ---------------------------------------------------------------------------
# minimal cell: 5 bohr square, 16 slices over 4 bohr, 6 random wells, V=0 leads
# ---------------------------------------------------------------------------
def minimal_cell(n_wells: int = 6, n_slices: int = 16, seed_cfg: int = 1,
                 energies=(0.5,), kpar=((0.0, 0.0),)) -> Instance:
    """Square 2D supercell a = 5 bohr, |G|^2 <= 5 (2 pi / a)^2 (21 vectors),
    device 4 bohr thick cut into equal slices, sum of Gaussian wells
    -V0 exp(-|r-R|^2 / 2 sigma^2), V0 ~ U[1,3] Ry, sigma = 0.6 bohr,
    centres uniform in the cell; V = 0 leads."""
    rng = _rng(seed_cfg)
    a = 5.0
    d = 4.0
    v0 = rng.uniform(1.0, 3.0, size=n_wells)
    pos = rng.uniform(0.0, 1.0, size=(n_wells, 3)) * np.array([a, a, d])
    b = 2.0 * math.pi / a
    e = np.asarray(energies, dtype=np.float64)
    k = np.asarray(kpar, dtype=np.float64).reshape(-1, 2)
    if len(k) == 1 and len(e) > 1:
        k = np.repeat(k, len(e), axis=0)
    if len(e) == 1 and len(k) > 1:
        e = np.repeat(e, len(k))
    return Instance(
        a1=np.array([a, 0.0]), a2=np.array([0.0, a]),
        ecut=5.0 * b * b * (1.0 + 1e-9), ng_exact=0,
        z_edges=np.linspace(0.0, d, n_slices + 1),
        wells_xyz=pos, v0=v0, sigma=np.full(n_wells, 0.6),
        lead_left=Lead.free(), lead_right=Lead.free(),
        energies=e, kpar=k, name="minimal_cell")


# ---------------------------------------------------------------------------
# graphene-like side-contact junction
# ---------------------------------------------------------------------------
def _sheet_cell_atoms(a: float) -> np.ndarray:
    """The 4 atoms (x, z) of one rectangular graphene cell a x sqrt(3) a with
    the zigzag direction along x: bond b = a / sqrt(3)."""
    b = a / math.sqrt(3.0)
    return np.array([[0.0, 0.0], [a / 2, b / 2], [a / 2, 3 * b / 2], [0.0, 2 * b]])


def junction(ng: int = 512, n_slices: int = 320, n_e: int = 128, n_k: int = 32,
             gap_angstrom: float = 3.35, stacking: str = "AB", v0: float = 2.0,
             sigma: float = 0.5, e_ref: float = 0.2, cells: int = 8,
             ecut: float | None = None, seed_cfg: int = 3) -> Instance:
    """Synthetic side-contact junction (the paper's Fig. 1 geometry with
    Gaussian carbon-like wells in place of DFT potentials).

    Transverse cell a_x = 2.46 A by L_y = 20 A (Sec. II B).  ``ng > 0`` takes
    the first ``ng`` G-vectors by (|G|^2, m, n); ``ng == 0`` uses the full
    shells below ``ecut``.  Energies are uniform in E_ref +- 2 eV; k_par runs
    on the line k_x = (2j - n_k + 1) pi / (n_k a_x), k_y = 0 (symmetric in +-k,
    containing neither 0 nor the zone edge).  The seed is unused (the junction
    is deterministic) but kept so that every instance is drawn the same way."""
    _rng(seed_cfg)
    ax = 2.46 * ANGSTROM
    ly = 20.0 * ANGSTROM
    cz = math.sqrt(3.0) * ax          # rectangular cell length along z
    lz = cells * cz
    gap = gap_angstrom * ANGSTROM
    cell = _sheet_cell_atoms(ax)
    shift = ax / math.sqrt(3.0) if stacking.upper() == "AB" else 0.0
    y_bot = ly / 2 - gap / 2
    y_top = ly / 2 + gap / 2
    bot_cells = range(0, cells - 2)
    top_cells = range(2, cells)
    wells = []
    for c in bot_cells:
        for (x, z) in cell:
            wells.append((x, y_bot, z + c * cz))
    for c in top_cells:
        for (x, z) in cell:
            wells.append((x, y_top, z + c * cz + shift))
    wells = np.array(wells)
    nw = len(wells)
    n_bot = len(bot_cells) * len(cell)
    rate = np.zeros((nw, 2))
    rate[:n_bot, 1] = -0.5          # y_bot = L_y/2 - gap/2
    rate[n_bot:, 1] = 0.5           # y_top = L_y/2 + gap/2
    lead_l = Lead(np.stack([cell[:, 0], np.full(4, y_bot)], axis=1),
                  np.full(4, v0), np.full(4, sigma), cz)
    lead_r = Lead(np.stack([cell[:, 0], np.full(4, y_top)], axis=1),
                  np.full(4, v0), np.full(4, sigma), cz)
    e = e_ref + (-2.0 + 4.0 * np.arange(n_e) / max(n_e - 1, 1)) / RYDBERG_EV
    kx = (2.0 * np.arange(n_k) - (n_k - 1)) * math.pi / (n_k * ax)
    ee, kk = np.meshgrid(e, kx, indexing="ij")
    # point order: k-major blocks (all energies of one k together)
    ee = ee.T.reshape(-1)
    kk = kk.T.reshape(-1)
    kpar = np.stack([kk, np.zeros_like(kk)], axis=1)
    return Instance(
        a1=np.array([ax, 0.0]), a2=np.array([0.0, ly]),
        ecut=(ecut if ecut is not None else 0.0), ng_exact=(ng if ecut is None else 0),
        z_edges=np.linspace(0.0, lz, n_slices + 1),
        wells_xyz=wells, v0=np.full(nw, v0), sigma=np.full(nw, sigma),
        lead_left=lead_l, lead_right=lead_r,
        energies=ee, kpar=kpar, name=f"junction_{stacking}_ng{ng}_ns{n_slices}",
        gap_rate_wells=rate, gap_rate_leads=np.array([[0.0, -0.5], [0.0, 0.5]]))


def uneven_batch(n_inst: int = 2048, ng_choices=tuple(range(128, 769, 64)), ns_range=(60, 400),
                 gap_range=(3.0, 5.0), e_ref: float = 0.2, seed_cfg: int = 4) -> list:
    """Independent junction instances of uneven size, one (E, k_par) point
    each: per instance (in this draw order) N_G uniform over ``ng_choices``,
    the slice count uniform in ``ns_range`` (inclusive), the gap uniform in
    ``gap_range`` (angstrom), AA or AB stacking with probability 1/2, E uniform
    in E_ref +- 2 eV and k_par uniform in the 2D Brillouin zone of the
    2.46 A x 20 A cell."""
    rng = _rng(seed_cfg)
    ax = 2.46 * ANGSTROM
    ly = 20.0 * ANGSTROM
    out = []
    for _ in range(n_inst):
        ng = int(rng.choice(np.asarray(ng_choices)))
        ns = int(rng.integers(ns_range[0], ns_range[1] + 1))
        gap = float(rng.uniform(*gap_range))
        stacking = "AB" if rng.uniform() < 0.5 else "AA"
        e = e_ref + float(rng.uniform(-2.0, 2.0)) / RYDBERG_EV
        k = np.array([rng.uniform(-math.pi / ax, math.pi / ax), rng.uniform(-math.pi / ly, math.pi / ly)])
        inst = junction(ng=ng, n_slices=ns, n_e=1, n_k=1, gap_angstrom=gap, stacking=stacking,
                        e_ref=e_ref, seed_cfg=seed_cfg)
        inst.energies = np.array([e])
        inst.kpar = k.reshape(1, 2)
        inst.name = f"uneven_{stacking}_ng{ng}_ns{ns}_gap{gap:.3f}"
        out.append(inst)
    return out


def junction_ecut_for(ng_full: int) -> float:
    """Cutoffs (Ry) whose full shells give the junction's odd N_G values."""
    return {401: 29.34, 513: 35.82}[ng_full]


def random_points(n: int, e_lo: float, e_hi: float, kmax: float, seed_cfg: int):
    """Uniform (E, k_par) draws: energies in [e_lo, e_hi), k in [-kmax, kmax)^2."""
    rng = _rng(seed_cfg)
    e = rng.uniform(e_lo, e_hi, size=n)
    k = rng.uniform(-kmax, kmax, size=(n, 2))
    return e, k


def explicit_barrier(v_slices, dz_slices, v_left=0.0, v_right=0.0, energies=(0.5,),
                     kpar=((0.0, 0.0),), a: float = 1.0) -> Instance:
    """A one-plane-wave (N_G = 1) instance given by explicit constant slice
    potentials: ``v_slices[p]`` is V^p(G=0), slice p has thickness
    ``dz_slices[p]``.  The cell is small enough that only G = 0 lies below the
    cutoff."""
    v = np.asarray(v_slices, dtype=np.float64)
    dz = np.asarray(dz_slices, dtype=np.float64)
    z = np.concatenate([[0.0], np.cumsum(dz)])
    b = 2 * math.pi / a
    tab = v.reshape(-1, 1, 1).astype(np.complex128)
    e = np.asarray(energies, dtype=np.float64)
    k = np.asarray(kpar, dtype=np.float64).reshape(-1, 2)
    if len(k) == 1 and len(e) > 1:
        k = np.repeat(k, len(e), axis=0)
    return Instance(
        a1=np.array([a, 0.0]), a2=np.array([0.0, a]), ecut=0.5 * b * b, ng_exact=0,
        z_edges=z, wells_xyz=np.zeros((0, 3)), v0=np.zeros(0), sigma=np.zeros(0),
        lead_left=Lead.free(), lead_right=Lead.free(), energies=e, kpar=k,
        slice_vg=tab,
        lead_vg=(np.array([[v_left]], dtype=np.complex128),
                 np.array([[v_right]], dtype=np.complex128)),
        vg_half=(0, 0), name="barrier")


def explicit_tables(a1, a2, ecut, z_edges, slice_vg, lead_l_vg, lead_r_vg, vg_half,
                    energies, kpar, ng_exact=0) -> Instance:
    """An instance given by explicit Fourier tables V^p(dG) indexed by
    (dm, dn) in [-Dm, Dm] x [-Dn, Dn] (``vg_half`` = (Dm, Dn)), stored as
    arrays of shape (n_slices, 2 Dm + 1, 2 Dn + 1); the lead tables share that
    shape (None = a V = 0 electrode)."""
    slice_vg = np.asarray(slice_vg, np.complex128)
    zero = np.zeros(slice_vg.shape[1:], np.complex128)
    lead_l_vg = zero if lead_l_vg is None else lead_l_vg
    lead_r_vg = zero if lead_r_vg is None else lead_r_vg
    return Instance(
        a1=np.asarray(a1, float), a2=np.asarray(a2, float), ecut=ecut, ng_exact=ng_exact,
        z_edges=np.asarray(z_edges, float), wells_xyz=np.zeros((0, 3)), v0=np.zeros(0),
        sigma=np.zeros(0), lead_left=Lead.free(), lead_right=Lead.free(),
        energies=np.asarray(energies, float), kpar=np.asarray(kpar, float).reshape(-1, 2),
        slice_vg=np.asarray(slice_vg, np.complex128),
        lead_vg=(np.asarray(lead_l_vg, np.complex128), np.asarray(lead_r_vg, np.complex128)),
        vg_half=tuple(vg_half), name="tables")


def random_tables(rng: np.random.Generator, n_slices: int, vg_half, scale: float,
                  decay: float = 0.5):
    """Random Hermitian-consistent Fourier tables V(-dG) = conj(V(dG)) for a real
    potential: draws only, indexed as in ``explicit_tables``."""
    dm, dn = vg_half
    shape = (n_slices, 2 * dm + 1, 2 * dn + 1)
    t = (rng.normal(size=shape) + 1j * rng.normal(size=shape)) * scale
    im = np.arange(-dm, dm + 1)[:, None]
    inn = np.arange(-dn, dn + 1)[None, :]
    t *= np.exp(-decay * (im ** 2 + inn ** 2))
    t = 0.5 * (t + np.conj(t[:, ::-1, ::-1]))
    return t
