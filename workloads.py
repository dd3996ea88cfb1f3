"""Seeded synthetic inputs for the RBSOG electrostatics path.

This module only builds particle systems (positions, charges, masses, LJ types,
molecules, bonds, angles and intramolecular exclusions).  It holds none of the
method's arithmetic, so that the CPU oracle (``oracle/``) and the CUDA path
(``paper_2602_23582_gb300``) can both be fed from it without sharing code.

Units are LAMMPS "real": Angstrom, g/mol, elementary charge, kcal/mol, radians.

The paper's own systems (SPC/E water with SHAKE, LiTFSI in TIP4P/2005 water,
a CHARMM36m DPPC membrane; paper section 4) are not available, so these
generators stand in for their shapes, sizes and charge/density structure:

* ``electrolyte``   1:1 point-charge electrolyte (1000 ions, 30 A box).
* ``water``         flexible 3-site SPC/E-charged water on a jittered lattice.
* ``ionic_liquid``  1-site cations + 15-site anions with random charges.
* ``membrane``      z-banded bilayer of +-0.5 dipolar pairs in water-like sites.
* ``served_batch``  many electrolyte/water systems of log-uniform size.
* ``nacl_crystal``  rock-salt supercell (Madelung test input).
* ``random_charges`` tiny neutral point-charge systems for brute-force tests.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "System", "electrolyte", "water", "ionic_liquid", "membrane",
    "served_batch", "nacl_crystal", "random_charges", "big_water",
]


@dataclasses.dataclass
class System:
    """One periodic orthorhombic particle system.

    ``mol`` gives every atom a molecule id; atoms of one molecule are
    contiguous and every single atom that is not part of a molecule has an id
    of its own.  ``excl`` lists every intramolecular pair (i < j): these pairs
    are left out of the short-range sums.
    """
    name: str
    pos: np.ndarray          # (N, 3) float64, inside [0, L)
    q: np.ndarray            # (N,) float64
    mass: np.ndarray         # (N,) float64
    type: np.ndarray         # (N,) int32
    mol: np.ndarray          # (N,) int32
    box: np.ndarray          # (3,) float64 edge lengths
    lj_eps: np.ndarray       # (T, T) float64
    lj_sig: np.ndarray       # (T, T) float64
    bonds: np.ndarray        # (nb, 2) int32
    bond_k: np.ndarray       # (nb,) float64, U = k (r - r0)^2
    bond_r0: np.ndarray      # (nb,) float64
    angles: np.ndarray       # (na, 3) int32, centre atom in the middle
    angle_k: np.ndarray      # (na,) float64, U = k (theta - theta0)^2
    angle_t0: np.ndarray     # (na,) float64
    excl: np.ndarray         # (ne, 2) int32
    coupling: int = 0        # 0 isotropic, 1 semi-isotropic (x=y coupled, z free)
    tilt: tuple = (0.0, 0.0, 0.0)   # (xy, xz, yz): h = [[Lx, xy, xz], [0, Ly, yz], [0, 0, Lz]]

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def ntypes(self) -> int:
        return int(self.lj_eps.shape[0])


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def _empty_i(shape):
    return np.zeros(shape, dtype=np.int32)


def _lj_table(eps, sig):
    """Lorentz-Berthelot mixing of per-type (eps, sigma)."""
    eps = np.asarray(eps, dtype=np.float64)
    sig = np.asarray(sig, dtype=np.float64)
    return np.sqrt(np.outer(eps, eps)), 0.5 * (sig[:, None] + sig[None, :])


def _random_rotations(rng, n):
    """Uniform random rotation matrices (unit quaternions, Shoemake)."""
    u1, u2, u3 = rng.random((3, n))
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    w = a * np.sin(2 * np.pi * u2)
    x = a * np.cos(2 * np.pi * u2)
    y = b * np.sin(2 * np.pi * u3)
    z = b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _intramolecular_pairs(mol_start, mol_size):
    """All i<j pairs inside each molecule (contiguous atom ranges)."""
    out = []
    for size in np.unique(mol_size):
        if size < 2:
            continue
        starts = mol_start[mol_size == size]
        ii, jj = np.triu_indices(size, k=1)
        out.append(np.stack([starts[:, None] + ii[None, :],
                             starts[:, None] + jj[None, :]], axis=-1).reshape(-1, 2))
    if not out:
        return _empty_i((0, 2))
    return np.concatenate(out).astype(np.int32)


def _close_pairs(pos, box, rmin):
    from scipy.spatial import cKDTree
    p = np.mod(pos, box)
    p[p >= box] = 0.0
    tree = cKDTree(p, boxsize=box)
    return tree.query_pairs(rmin, output_type="ndarray")


def _random_packing(rng, n, box, min_dist, batch=4096):
    """Random sequential insertion in batches: a uniform candidate is
    dropped when it lies within ``min_dist`` (minimum image) of a point kept
    earlier or of an earlier candidate of its own batch."""
    from scipy.spatial import cKDTree
    box = np.asarray(box, dtype=np.float64)
    kept = np.empty((0, 3))
    for _ in range(100000):
        if len(kept) >= n:
            break
        cand = rng.random((min(batch, 4 * (n - len(kept)) + 16), 3)) * box
        cand[cand >= box] = 0.0
        if len(kept):
            d, _ = cKDTree(kept, boxsize=box).query(cand, k=1)
            cand = cand[d >= min_dist]
        acc = []
        if len(cand):
            pairs = cKDTree(cand, boxsize=box).query_pairs(min_dist, output_type="ndarray")
            taken = np.ones(len(cand), bool)
            if len(pairs):
                taken[pairs.max(axis=1)] = False
            acc = cand[taken]
        if len(acc):
            kept = np.concatenate([kept, acc])
    if len(kept) < n:
        raise RuntimeError("packing failed")
    return kept[:n]


def _water_frame(theta0_deg=109.47, r_oh=1.0):
    """O at the origin, both H in the xz-plane, bisector along +z."""
    half = math.radians(theta0_deg) / 2
    return np.array([[0.0, 0.0, 0.0],
                     [r_oh * math.sin(half), 0.0, r_oh * math.cos(half)],
                     [-r_oh * math.sin(half), 0.0, r_oh * math.cos(half)]])


# SPC/E charges and LJ; SPC/Fw-like flexible force constants (U = k (x - x0)^2).
_SPCE_QO, _SPCE_QH = -0.8476, 0.4238
_SPCE_SIG_O, _SPCE_EPS_O = 3.166, 0.1553
_WATER_KB, _WATER_R0 = 529.581, 1.0
_WATER_KA, _WATER_T0 = 37.95, math.radians(109.47)
_M_O, _M_H = 15.9994, 1.008


def _water_block(centres, R, atom0, mol0):
    """3-site molecules at ``centres`` (O) with orientation matrices ``R``."""
    nm = centres.shape[0]
    frame = _water_frame()
    sites = centres[:, None, :] + np.einsum("nij,sj->nsi", R, frame)
    pos = sites.reshape(-1, 3)
    q = np.tile([_SPCE_QO, _SPCE_QH, _SPCE_QH], nm)
    mass = np.tile([_M_O, _M_H, _M_H], nm)
    mol = np.repeat(np.arange(mol0, mol0 + nm, dtype=np.int32), 3)
    base = atom0 + 3 * np.arange(nm, dtype=np.int32)
    bonds = np.concatenate([np.stack([base, base + 1], 1), np.stack([base, base + 2], 1)])
    angles = np.stack([base + 1, base, base + 2], 1)
    return pos, q, mass, mol, bonds.astype(np.int32), angles.astype(np.int32)


def _finish(name, pos, q, mass, typ, mol, box, eps, sig, bonds=None, bond_k=None,
            bond_r0=None, angles=None, angle_k=None, angle_t0=None, coupling=0):
    box = np.asarray(box, dtype=np.float64)
    pos = np.mod(np.asarray(pos, dtype=np.float64), box)
    pos[pos >= box] = 0.0
    mol = np.asarray(mol, dtype=np.int32)
    # molecule extents (contiguous)
    change = np.flatnonzero(np.diff(mol)) + 1
    starts = np.concatenate([[0], change]).astype(np.int64)
    sizes = np.diff(np.concatenate([starts, [mol.size]]))
    if np.unique(mol[starts]).size != starts.size:
        raise ValueError("molecules must be contiguous")
    nb = 0 if bonds is None else len(bonds)
    na = 0 if angles is None else len(angles)
    lj_eps, lj_sig = _lj_table(eps, sig)
    return System(
        name=name, pos=pos, q=np.asarray(q, dtype=np.float64),
        mass=np.asarray(mass, dtype=np.float64), type=np.asarray(typ, dtype=np.int32),
        mol=mol, box=box, lj_eps=lj_eps, lj_sig=lj_sig,
        bonds=_empty_i((0, 2)) if nb == 0 else np.asarray(bonds, dtype=np.int32),
        bond_k=np.zeros(0) if nb == 0 else np.asarray(bond_k, dtype=np.float64),
        bond_r0=np.zeros(0) if nb == 0 else np.asarray(bond_r0, dtype=np.float64),
        angles=_empty_i((0, 3)) if na == 0 else np.asarray(angles, dtype=np.int32),
        angle_k=np.zeros(0) if na == 0 else np.asarray(angle_k, dtype=np.float64),
        angle_t0=np.zeros(0) if na == 0 else np.asarray(angle_t0, dtype=np.float64),
        excl=_intramolecular_pairs(starts, sizes), coupling=coupling)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def electrolyte(n_ions: int = 1000, L: float = 30.0, seed: int = 1,
                min_dist: float = 2.5) -> System:
    """1:1 point-charge electrolyte: n/2 cations (+1) and n/2 anions (-1),
    uniform random in a cube by batched random sequential insertion, a
    candidate rejected when it comes closer than ``min_dist`` (minimum image)
    to an ion already placed.  LJ sigma 3 A,
    epsilon 0.1 kcal/mol on both species; masses 22.99 / 35.45 g/mol."""
    rng = np.random.default_rng(seed)
    box = np.array([L, L, L])
    pos = _random_packing(rng, n_ions, box, min_dist)
    half = n_ions // 2
    q = np.concatenate([np.ones(half), -np.ones(n_ions - half)])
    typ = np.concatenate([np.zeros(half, np.int32), np.ones(n_ions - half, np.int32)])
    mass = np.where(typ == 0, 22.99, 35.45)
    mol = np.arange(n_ions, dtype=np.int32)
    return _finish("electrolyte", pos, q, mass, typ, mol, box, [0.1, 0.1], [3.0, 3.0])


def water(n_mol: int = 10000, L: float = 66.88, seed: int = 2, lattice: int = 22,
          jitter: float = 0.2) -> System:
    """Flexible 3-site water with SPC/E charges (-0.8476/+0.4238) and geometry
    (O-H 1 A, H-O-H 109.47 deg): O on a jittered simple-cubic lattice of
    ``lattice``^3 sites (the first ``n_mol`` used), random orientations.
    1 g/cm^3 at 10,000 molecules gives L = 66.88 A."""
    rng = np.random.default_rng(seed)
    if lattice ** 3 < n_mol:
        raise ValueError("lattice too small")
    a = L / lattice
    g = np.arange(lattice)
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)[:n_mol]
    centres = (grid + 0.5) * a + rng.uniform(-jitter, jitter, (n_mol, 3))
    R = _random_rotations(rng, n_mol)
    pos, q, mass, mol, bonds, angles = _water_block(centres, R, 0, 0)
    typ = np.tile(np.array([0, 1, 1], np.int32), n_mol)
    nb, na = len(bonds), len(angles)
    return _finish("water", pos, q, mass, typ, mol, [L, L, L],
                   [_SPCE_EPS_O, 0.0], [_SPCE_SIG_O, 1.0],
                   bonds, np.full(nb, _WATER_KB), np.full(nb, _WATER_R0),
                   angles, np.full(na, _WATER_KA), np.full(na, _WATER_T0))


def big_water(n_sites: int = 10_000_000, seed: int = 6, min_contact: float = 0.8) -> System:
    """The 10^7-site water-like scale point: ceil(n_sites/3) molecules at
    1 g/cm^3 (L = 463.7 A for 3,333,334 molecules), jittered lattice, random
    orientations redrawn (all at once per round) for every molecule with a
    site closer than ``min_contact`` to another molecule's site: among 3.3e6
    random orientations some O-H contacts come out far closer than any in the
    10,000-molecule box (0.80 A there, which runs stably), and H carries no LJ
    core to stop them collapsing."""
    from scipy.spatial import cKDTree
    n_mol = -(-n_sites // 3)
    L = 66.88 * (n_mol / 10000.0) ** (1.0 / 3.0)
    lattice = int(math.ceil(n_mol ** (1.0 / 3.0)))
    rng = np.random.default_rng(seed)
    a = L / lattice
    g = np.arange(lattice)
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)[:n_mol]
    centres = (grid + 0.5) * a + rng.uniform(-0.2, 0.2, (n_mol, 3))
    R = _random_rotations(rng, n_mol)
    frame = _water_frame()
    sites = centres[:, None, :] + np.einsum("nij,sj->nsi", R, frame)
    box = np.array([L, L, L])
    for _ in range(100):
        p = np.mod(sites.reshape(-1, 3), box)
        p[p >= box] = 0.0
        pairs = cKDTree(p, boxsize=box).query_pairs(min_contact, output_type="ndarray") // 3
        bad = np.unique(pairs[pairs[:, 0] != pairs[:, 1]])
        if bad.size == 0:
            break
        R[bad] = _random_rotations(rng, bad.size)
        sites[bad] = centres[bad][:, None, :] + np.einsum("nij,sj->nsi", R[bad], frame)
    else:
        raise RuntimeError("could not remove close contacts")
    pos, q, mass, mol, bonds, angles = _water_block(centres, R, 0, 0)
    typ = np.tile(np.array([0, 1, 1], np.int32), n_mol)
    nb, na = len(bonds), len(angles)
    return _finish("water", pos, q, mass, typ, mol, box,
                   [_SPCE_EPS_O, 0.0], [_SPCE_SIG_O, 1.0],
                   bonds, np.full(nb, _WATER_KB), np.full(nb, _WATER_R0),
                   angles, np.full(na, _WATER_KA), np.full(na, _WATER_T0))


def _anion_template(rng, n_sites=15, radius=3.5, dmin=1.2):
    pts = [np.zeros(3)]
    while len(pts) < n_sites:
        c = rng.uniform(-radius, radius, 3)
        if np.linalg.norm(c) > radius:
            continue
        if min(np.linalg.norm(c - p) for p in pts) < dmin:
            continue
        pts.append(c)
    pts = np.array(pts)
    return pts - pts.mean(0)


def _fix_overlaps(pos, mol_of, mol_start, mol_size, centres, frames, R, box, rng,
                  rmin, rounds=200):
    """Re-draw the orientation of molecules that hold a site closer than
    ``rmin`` to another molecule's site, until none is left."""
    for _ in range(rounds):
        pairs = _close_pairs(pos, box, rmin)
        if len(pairs):
            pairs = pairs[mol_of[pairs[:, 0]] != mol_of[pairs[:, 1]]]
        if not len(pairs):
            return pos
        bad = np.unique(mol_of[pairs.reshape(-1)])
        R[bad] = _random_rotations(rng, bad.size)
        single = bad[mol_size[bad] == 1]
        centres[single] += rng.uniform(-0.5, 0.5, (single.size, 3))
        for m in bad:
            s, n = mol_start[m], mol_size[m]
            pos[s:s + n] = centres[m] + frames[m] @ R[m].T
    raise RuntimeError("could not remove overlaps")


def ionic_liquid(n_pairs: int = 4000, seed: int = 3, density: float = 1.4,
                 n_anion_sites: int = 15) -> System:
    """4,000 one-site cations (+1, 6.94 g/mol) and 4,000 rigid-geometry
    15-site anions (280.15 g/mol spread evenly), 64,000 sites.  One random
    template (sites >= 1.2 A apart within 3.5 A); per anion, charges drawn
    uniform in [-0.6, 0.6], shifted to sum to -1 and redrawn while any
    |q| > 0.6.  The anion's geometry is held by harmonic springs between every
    template site pair closer than 3 A.  Molecules sit on a jittered rock-salt
    lattice (anions on one sublattice) with random orientations; orientations are redrawn while sites of two
    molecules come closer than 1.2 A.  1.4 g/cm^3 gives L = 110.85 A."""
    rng = np.random.default_rng(seed)
    m_cat, m_an = 6.94, 280.15
    total_mass = n_pairs * (m_cat + m_an)
    V = total_mass / (0.602214076 * density)          # A^3
    L = V ** (1.0 / 3.0)
    box = np.array([L, L, L])
    tmpl = _anion_template(rng, n_anion_sites)
    n_mol = 2 * n_pairs
    lat = int(math.ceil(n_mol ** (1.0 / 3.0)))
    a = L / lat
    g = np.arange(lat)
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    # rock-salt ordering of the two species keeps anions off neighbouring sites
    even = grid.sum(1) % 2 == 0
    an_sites = grid[even][rng.permutation(int(even.sum()))[:n_pairs]]
    cat_sites = grid[~even][rng.permutation(int((~even).sum()))[:n_pairs]]
    grid = np.concatenate([an_sites, cat_sites])
    order = rng.permutation(n_mol)
    grid = grid[order]
    is_anion = order < n_pairs
    centres = (grid + 0.5) * a + rng.uniform(-0.3, 0.3, (n_mol, 3))
    sizes = np.where(is_anion, n_anion_sites, 1)
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    N = int(sizes.sum())
    frames = [tmpl if an else np.zeros((1, 3)) for an in is_anion]
    R = _random_rotations(rng, n_mol)
    pos = np.empty((N, 3))
    q = np.empty(N)
    mass = np.empty(N)
    typ = np.empty(N, np.int32)
    mol_of = np.repeat(np.arange(n_mol, dtype=np.int32), sizes)
    for m in range(n_mol):
        s, n = starts[m], sizes[m]
        pos[s:s + n] = centres[m] + frames[m] @ R[m].T
        if is_anion[m]:
            while True:
                qq = rng.uniform(-0.6, 0.6, n)
                qq += (-1.0 - qq.sum()) / n
                if np.all(np.abs(qq) <= 0.6):
                    break
            q[s:s + n] = qq
            mass[s:s + n] = m_an / n
            typ[s:s + n] = 1
        else:
            q[s] = 1.0
            mass[s] = m_cat
            typ[s] = 0
    pos = _fix_overlaps(pos, mol_of, starts, sizes, centres, frames, R, box, rng, 1.2)
    ti, tj = np.triu_indices(n_anion_sites, 1)
    d = np.linalg.norm(tmpl[ti] - tmpl[tj], axis=1)
    keep = d < 3.0
    an_starts = starts[is_anion]
    bonds = np.stack([an_starts[:, None] + ti[keep][None, :],
                      an_starts[:, None] + tj[keep][None, :]], -1).reshape(-1, 2)
    r0 = np.tile(d[keep], n_pairs)
    return _finish("ionic_liquid", pos, q, mass, typ, mol_of, box, [0.1, 0.1], [3.0, 3.0],
                   bonds, np.full(len(bonds), 100.0), r0)


def membrane(seed: int = 4, Lxy: float = 64.0, Lz: float = 96.0,
             n_sites: int = 120_000, band_half: float = 20.0,
             lattice=(43, 43, 65), jitter: float = 0.1) -> System:
    """Membrane-shaped anisotropic slab, 64 x 64 x 96 A with 120,000 sites
    (0.305 A^-3, about 3x liquid water, so molecules cannot be placed with
    free orientations).  Every site sits on a jittered 43 x 43 x 65 lattice
    (spacing ~1.48 A):

    * band |z - Lz/2| <= 20 A: +-0.5 dipolar pairs made of two z-adjacent
      sites (1.48 A apart, along +z or -z at random, tilted by the jitter);
    * the rest: 3-site water-like molecules (-0.8476 centre, +0.4238 ends)
      made of three consecutive sites of a snake path through the lattice,
      held by harmonic springs (centre-end and end-end) whose equilibrium
      lengths are the initial ones.

    185 lattice sites stay empty.  LJ sigma 2 A, epsilon 0.1 kcal/mol on every
    site (a 3 A sigma cannot fit this density).  Semi-isotropic coupling."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = lattice
    box = np.array([Lxy, Lxy, Lz])
    a = box / np.array(lattice)
    zc = (np.arange(nz) + 0.5) * a[2]
    band_layers = np.flatnonzero(np.abs(zc - Lz / 2) <= band_half)
    if band_layers.size % 2:
        band_layers = band_layers[:-1]
    n_col = nx * ny
    n_dip = (band_layers.size // 2) * n_col
    while (n_sites - 2 * n_dip) % 3:
        n_dip -= 1
    n_wat = (n_sites - 2 * n_dip) // 3
    # dipoles: columns of each band layer pair
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    ii, jj = ii.reshape(-1), jj.reshape(-1)
    dip_sites = []
    for p in range(band_layers.size // 2):
        k0 = band_layers[2 * p]
        lo = np.stack([ii, jj, np.full(n_col, k0)], 1)
        hi = np.stack([ii, jj, np.full(n_col, k0 + 1)], 1)
        dip_sites.append(np.stack([lo, hi], 1))
    dip_sites = np.concatenate(dip_sites)[:n_dip]               # (n_dip, 2, 3)
    flip = rng.random(n_dip) < 0.5
    dip_sites[flip] = dip_sites[flip][:, ::-1]
    # water: snake through the remaining layers, starting above the band
    wl = [k for k in range(band_layers[-1] + 1, nz)] + [k for k in range(0, band_layers[0])]
    snake = []
    for n_l, k in enumerate(wl):
        for j_idx in range(ny):
            j = j_idx if n_l % 2 == 0 else ny - 1 - j_idx
            row = np.arange(nx) if (j_idx % 2 == 0) else np.arange(nx)[::-1]
            snake.append(np.stack([row, np.full(nx, j), np.full(nx, k)], 1))
    snake = np.concatenate(snake)[:3 * n_wat].reshape(n_wat, 3, 3)
    grid = np.concatenate([dip_sites.reshape(-1, 3), snake.reshape(-1, 3)])
    pos = (grid + 0.5) * a + rng.uniform(-jitter, jitter, grid.shape)
    N = pos.shape[0]
    assert N == n_sites
    q = np.concatenate([np.tile([-0.5, 0.5], n_dip), np.tile([_SPCE_QO, _SPCE_QH, _SPCE_QH], n_wat)])
    mass = np.concatenate([np.full(2 * n_dip, 12.0), np.tile([_M_O, _M_H, _M_H], n_wat)])
    sizes = np.concatenate([np.full(n_dip, 2), np.full(n_wat, 3)])
    mol_of = np.repeat(np.arange(n_dip + n_wat, dtype=np.int32), sizes)
    # water: centre site (O) first in storage order: reorder snake triple (e, c, e) -> (c, e, e)
    wbase = 2 * n_dip + 3 * np.arange(n_wat)
    wp = pos[2 * n_dip:].reshape(n_wat, 3, 3)[:, [1, 0, 2]]
    pos[2 * n_dip:] = wp.reshape(-1, 3)

    def mi(d):
        return d - box * np.rint(d / box)
    d1 = mi(wp[:, 1] - wp[:, 0])
    d2 = mi(wp[:, 2] - wp[:, 0])
    r1 = np.linalg.norm(d1, axis=1)
    r2 = np.linalg.norm(d2, axis=1)
    dip_b = 2 * np.arange(n_dip)
    dd = np.linalg.norm(mi(pos[dip_b + 1] - pos[dip_b]), axis=1)
    typ = np.zeros(N, np.int32)
    r12 = np.linalg.norm(mi(wp[:, 2] - wp[:, 1]), axis=1)
    # the snake makes some triples straight, where a harmonic angle term is
    # singular; the end-to-end spring holds the shape instead (no angles)
    bonds = np.concatenate([np.stack([dip_b, dip_b + 1], 1),
                            np.stack([wbase, wbase + 1], 1), np.stack([wbase, wbase + 2], 1),
                            np.stack([wbase + 1, wbase + 2], 1)])
    bk = np.concatenate([np.full(n_dip, 450.0), np.full(2 * n_wat, _WATER_KB),
                         np.full(n_wat, 50.0)])
    br = np.concatenate([dd, r1, r2, r12])
    return _finish("membrane", pos, q, mass, typ, mol_of, box, [0.1], [2.0],
                   bonds, bk, br, coupling=1)


def served_batch(n_systems: int = 256, seed: int = 5, n_min: int = 500,
                 n_max: int = 20000, min_box: float = 28.0, steps=(100, 1000),
                 rate_per_ms: float | None = None, workers: int = 1):
    """Served-request stream: ``n_systems`` independent systems, sizes
    log-uniform in [n_min, n_max] sites, each an electrolyte (C1 density) or a
    water-like box (1 g/cm^3) at random.  A system whose box at that density
    would be shorter than ``min_box`` (28 A: the 5 x 5 x 5 stencil of cells of
    r_c / 2 at r_c = 10 A needs 25 A, and the box breathes under NPT) is given
    more atoms, at the same density, to fill a box of ``min_box`` (a box
    widened at a fixed atom count would be dilute, and collapse under 1 atm
    below the stencil's size).  Each request
    asks for a uniform number of NPT steps in ``steps``; arrivals are a
    Poisson stream of ``rate_per_ms`` requests per millisecond (all at t=0
    when None).  ``workers`` > 1 builds the systems in that many spawned
    processes (same systems).  Returns a list of (arrival_ms, n_steps, System)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_systems))
    kinds = rng.random(n_systems) < 0.5
    nsteps = rng.integers(steps[0], steps[1] + 1, n_systems)
    if rate_per_ms:
        t = np.cumsum(rng.exponential(1.0 / rate_per_ms, n_systems))
    else:
        t = np.zeros(n_systems)
    jobs = [(bool(kinds[i]), float(sizes[i]), int(rng.integers(1 << 30)), float(min_box)) for i in range(n_systems)]
    if workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            systems = list(ex.map(_served_system, jobs, chunksize=4))
    else:
        systems = [_served_system(j) for j in jobs]
    return [(float(t[i]), int(nsteps[i]), systems[i]) for i in range(n_systems)]


def _served_system(job):
    """One system of the served stream: (electrolyte?, size, seed, min box)."""
    is_el, size, sub, min_box = job
    if is_el:
        rho = 1000 / 27000.0                            # the C1 electrolyte's ions per A^3
        n = max(2, int(round(size / 2)) * 2)
        n = max(n, 2 * int(math.ceil(rho * min_box ** 3 / 2)))
        L = (n / rho) ** (1 / 3)
        return electrolyte(n, L, seed=sub, min_dist=min(2.5, 0.8 * L / n ** (1 / 3)))
    nm = max(1, int(round(size / 3)))
    nm = max(nm, int(math.ceil(10000.0 * (min_box / 66.88) ** 3)))
    L = 66.88 * (nm / 10000.0) ** (1 / 3)
    lat = int(math.ceil(nm ** (1 / 3)))
    return water(nm, L, seed=sub, lattice=lat)


def nacl_crystal(cells: int = 4, a: float = 5.64) -> System:
    """Rock-salt supercell of ``cells``^3 conventional cells (8 ions each)."""
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.arange(cells)
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    na = (grid[:, None, :] + base[None, :, :]).reshape(-1, 3)
    cl = (grid[:, None, :] + base[None, :, :] + np.array([0.5, 0, 0])).reshape(-1, 3)
    pos = np.concatenate([na, cl]) * a
    n = pos.shape[0]
    q = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    typ = np.concatenate([np.zeros(n // 2, np.int32), np.ones(n // 2, np.int32)])
    L = cells * a
    return _finish("nacl", pos, q, np.where(typ == 0, 22.99, 35.45), typ,
                   np.arange(n, dtype=np.int32), [L, L, L], [0.0, 0.0], [1.0, 1.0])


def sheared(sys: System, tilt) -> System:
    """The same system in a triclinic cell: edge lengths kept, tilts (xy, xz,
    yz) added.  Each molecule moves rigidly so that its first atom keeps its
    fractional coordinates (s = r / L of the orthorhombic box, r' = h s), then
    every atom is wrapped into the cell by whole cell vectors; intramolecular
    geometry is unchanged."""
    L = np.asarray(sys.box, dtype=np.float64)
    xy, xz, yz = (float(t) for t in tilt)
    h = np.array([[L[0], xy, xz], [0.0, L[1], yz], [0.0, 0.0, L[2]]])
    pos = np.array(sys.pos, dtype=np.float64)
    change = np.flatnonzero(np.diff(sys.mol)) + 1
    starts = np.concatenate([[0], change]).astype(np.int64)
    ends = np.concatenate([change, [sys.n]]).astype(np.int64)
    for a, b in zip(starts, ends):
        d = pos[a:b] - pos[a]
        d -= L * np.rint(d / L)                  # the molecule whole (minimum image in the old box)
        pos[a:b] = h @ (pos[a] / L) + d
    sfrac = np.linalg.solve(h, pos.T).T
    pos -= np.floor(sfrac) @ h.T
    out = dataclasses.replace(sys, pos=pos, tilt=(xy, xz, yz), coupling=2)
    return out


def random_charges(n: int = 64, box=(20.0, 20.0, 20.0), seed: int = 0,
                   min_dist: float = 1.5, lj: bool = False, qmax: float = 1.0) -> System:
    """Tiny neutral system: n random charges (uniform in [-qmax, qmax], the
    last one set to make the total zero), uniform positions with a minimum
    image spacing of ``min_dist``."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    pos = _random_packing(rng, n, box, min_dist)
    q = rng.uniform(-qmax, qmax, n)
    q -= q.mean()
    typ = np.zeros(n, np.int32)
    eps = [0.1] if lj else [0.0]
    return _finish("random", pos, q, np.full(n, 20.0), typ,
                   np.arange(n, dtype=np.int32), box, eps, [2.5])
