"""Seeded synthetic inputs: molecular geometries, contracted Gaussian basis sets
and distance-decaying density matrices.

This module is shared by the CPU oracle tests, the GPU parity tests and the
benchmark. It holds only input generation: geometry construction, random
exponents/coefficients for contracted shells and the density recipe. It holds
none of the Fock-build arithmetic (no normalisation, no integrals, no
screening), so neither side of a parity comparison can inherit a mistake from
the other through it.

Units: geometries are built in Angstrom and returned in bohr
(1 bohr = 0.529177210903 Angstrom, CODATA 2018); exponents are in bohr^-2.

Shell layout returned by :func:`make_basis` (all numpy arrays):

- ``center``  float64 [nshell, 3]  shell centre (bohr)
- ``l``       int32   [nshell]     angular momentum 0..3
- ``nprim``   int32   [nshell]     contraction length K
- ``prim_off``int32   [nshell]     offset of the shell's primitives in exps/coefs
- ``exps``    float64 [nprimtot]   exponents alpha_k = a0 * b**k
- ``coefs``   float64 [nprimtot]   raw contraction coefficients of
                                   primitive-normalised Gaussians (positive)
- ``atom``    int32   [nshell]     index of the atom carrying the shell

Cartesian functions of a shell follow the order x^l, x^(l-1)y, x^(l-1)z, ...,
z^l (exponent of x descending, then y descending).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BOHR_ANGSTROM = 0.529177210903

# Shell recipes: (l, K) per shell, in the order they are attached to an atom.
# "dz": 6-31G(d)-shaped; heavy atoms O/C share the same shape.
DZ_HEAVY = [(0, 6), (0, 3), (1, 3), (0, 1), (1, 1), (2, 1)]
DZ_H = [(0, 3), (0, 1)]
# "tz": triple-zeta-shaped, highly contracted, up to f.
TZ_HEAVY = [(0, 8), (0, 3), (0, 1), (0, 1), (1, 4), (1, 1), (1, 1), (2, 1), (2, 1), (3, 1)]
TZ_H = [(0, 5), (0, 1), (0, 1), (1, 1)]

ELEMENT_Z = {"H": 1, "C": 6, "O": 8}


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


@dataclass
class Molecule:
    symbols: list
    coords: np.ndarray  # [natom, 3] bohr

    @property
    def natom(self) -> int:
        return len(self.symbols)

    @property
    def Z(self) -> np.ndarray:
        return np.array([ELEMENT_Z[s] for s in self.symbols], dtype=np.int32)


@dataclass
class Problem:
    name: str
    mol: Molecule
    basis: dict
    D: np.ndarray
    tau: float
    meta: dict = field(default_factory=dict)

    @property
    def nbf(self) -> int:
        return self.D.shape[0]


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------

def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly distributed rotation matrix (QR of a Gaussian matrix, sign-fixed)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def water_molecule(rng: np.random.Generator, o_pos_ang: np.ndarray) -> np.ndarray:
    """O-H 0.96 A, H-O-H 104.5 deg, uniformly random orientation; Angstrom."""
    half = math.radians(104.5) / 2.0
    r = 0.96
    local = np.array([[0.0, 0.0, 0.0],
                      [r * math.sin(half), 0.0, r * math.cos(half)],
                      [-r * math.sin(half), 0.0, r * math.cos(half)]])
    rot = random_rotation(rng)
    return local @ rot.T + o_pos_ang[None, :]


def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def water_chain_cluster(n: int, rng: np.random.Generator, dmin=2.8, dmax=3.2) -> Molecule:
    """Waters placed one by one, each new O at dmin..dmax A from a random existing O,
    rejecting any O-O distance below dmin."""
    oxy = [np.zeros(3)]
    tries = 0
    while len(oxy) < n:
        tries += 1
        if tries > 100000:
            raise RuntimeError("water placement failed")
        base = oxy[rng.integers(len(oxy))]
        cand = base + random_unit(rng) * rng.uniform(dmin, dmax)
        if min(np.linalg.norm(cand - o) for o in oxy) < dmin - 1e-12:
            continue
        oxy.append(cand)
    syms, xyz = [], []
    for o in oxy:
        w = water_molecule(rng, o)
        syms += ["O", "H", "H"]
        xyz.append(w)
    return Molecule(syms, np.concatenate(xyz) / BOHR_ANGSTROM)


def water_sphere_cluster(n: int, rng: np.random.Generator, density=0.033, dmin=2.6) -> Molecule:
    """n waters with O uniform in a sphere at the given number density
    (molecules / A^3), rejecting O-O closer than dmin A; random orientations."""
    radius = (3.0 * n / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    oxy = []
    tries = 0
    while len(oxy) < n:
        tries += 1
        if tries > 5_000_000:
            raise RuntimeError("water sphere packing failed")
        p = rng.uniform(-radius, radius, 3)
        if np.linalg.norm(p) > radius:
            continue
        if oxy and min(np.linalg.norm(p - o) for o in oxy) < dmin:
            continue
        oxy.append(p)
    syms, xyz = [], []
    for o in oxy:
        syms += ["O", "H", "H"]
        xyz.append(water_molecule(rng, o))
    return Molecule(syms, np.concatenate(xyz) / BOHR_ANGSTROM)


def alkane_zigzag(nc: int, cc=1.54, ch=1.09, torsions=None, rng=None) -> Molecule:
    """C_nH_(2n+2) in the all-trans zigzag (torsions=None) or with the given
    C-C-C-C torsion angles (radians, length nc-3). Tetrahedral angles throughout."""
    tet = math.acos(-1.0 / 3.0)
    # backbone
    c = [np.zeros(3)]
    if nc >= 2:
        c.append(np.array([cc, 0.0, 0.0]))
    if nc >= 3:
        ang = math.pi - tet
        c.append(c[1] + cc * np.array([math.cos(ang), math.sin(ang), 0.0]))
    for i in range(3, nc):
        phi = math.pi if torsions is None else float(torsions[i - 3])
        c.append(_place_dihedral(c[i - 3], c[i - 2], c[i - 1], cc, tet, phi))
    syms = ["C"] * nc
    hs = []
    for i in range(nc):
        nbr = []
        if i > 0:
            nbr.append(c[i - 1])
        if i + 1 < nc:
            nbr.append(c[i + 1])
        hs += _hydrogens(c[i], nbr, 4 - len(nbr), ch, tet, c, i)
    xyz = np.array(c + hs)
    syms += ["H"] * len(hs)
    return Molecule(syms, xyz / BOHR_ANGSTROM)


def _place_dihedral(a, b, c, bond, angle, dihedral):
    bc = c - b
    bc /= np.linalg.norm(bc)
    n = np.cross(b - a, bc)
    n /= np.linalg.norm(n)
    m = np.cross(n, bc)
    d2 = np.array([-bond * math.cos(angle),
                   bond * math.sin(angle) * math.cos(dihedral),
                   bond * math.sin(angle) * math.sin(dihedral)])
    return c + d2[0] * bc + d2[1] * m + d2[2] * n


def _hydrogens(ci, nbr, nh, ch, tet, chain, i):
    """Tetrahedral H positions around carbon ci with the given carbon neighbours."""
    if len(nbr) == 0:  # methane
        dirs = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) / math.sqrt(3)
        return [ci + ch * d for d in dirs]
    if len(nbr) == 2:
        u1 = (nbr[0] - ci) / np.linalg.norm(nbr[0] - ci)
        u2 = (nbr[1] - ci) / np.linalg.norm(nbr[1] - ci)
        bis = -(u1 + u2)
        bis /= np.linalg.norm(bis)
        perp = np.cross(u1, u2)
        perp /= np.linalg.norm(perp)
        h = tet / 2.0
        return [ci + ch * (bis * math.cos(h) + s * perp * math.sin(h)) for s in (1.0, -1.0)]
    # terminal carbon: one neighbour; three H staggered about the C-C axis
    u = (ci - nbr[0]) / np.linalg.norm(ci - nbr[0])
    ref = None
    j = i - 1 if i > 0 else i + 1
    k = j - 1 if i > 0 else j + 1
    if 0 <= k < len(chain):
        ref = chain[k] - chain[j]
    if ref is None or np.linalg.norm(np.cross(ref, u)) < 1e-8:
        ref = np.array([0.0, 0.0, 1.0]) if abs(u[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    w = ref - np.dot(ref, u) * u
    w /= np.linalg.norm(w)
    v = np.cross(u, w)
    out = []
    for kk in range(3):
        phi = math.pi + 2.0 * math.pi * kk / 3.0
        d = u * (-math.cos(tet)) + math.sin(tet) * (math.cos(phi) * w + math.sin(phi) * v)
        out.append(ci + ch * d / np.linalg.norm(d))
    return out[:3]


def combine(*mols: Molecule) -> Molecule:
    return Molecule(sum((m.symbols for m in mols), []), np.concatenate([m.coords for m in mols]))


# ----------------------------------------------------------------------------
# basis
# ----------------------------------------------------------------------------

def element_basis(rng: np.random.Generator, recipe) -> list:
    """Random shells for one element: alpha_k = a0*b**k, a0~U[0.1,0.3], b~U[2.5,4],
    raw coefficients ~U[0.1,1]. Returns [(l, exps, coefs)]."""
    shells = []
    for l, K in recipe:
        a0 = rng.uniform(0.1, 0.3)
        b = rng.uniform(2.5, 4.0)
        exps = a0 * b ** np.arange(K, dtype=np.float64)
        coefs = rng.uniform(0.1, 1.0, K)
        shells.append((l, exps[::-1].copy(), coefs[::-1].copy()))
    return shells


def basis_set(kind: str, seed: int) -> dict:
    """Per-element basis table {symbol: [(l, exps, coefs)]} drawn from a seed."""
    rng = np.random.Generator(np.random.PCG64(10_000 + seed))
    heavy, light = (DZ_HEAVY, DZ_H) if kind == "dz" else (TZ_HEAVY, TZ_H)
    table = {}
    heavy_shells = element_basis(rng, heavy)
    table["O"] = heavy_shells
    table["C"] = element_basis(rng, heavy)
    table["H"] = element_basis(rng, light)
    return table


def make_basis(mol: Molecule, table: dict) -> dict:
    center, ls, nprim, off, exps, coefs, atom = [], [], [], [], [], [], []
    n = 0
    for ia, (sym, xyz) in enumerate(zip(mol.symbols, mol.coords)):
        for l, e, c in table[sym]:
            center.append(xyz)
            ls.append(l)
            nprim.append(len(e))
            off.append(n)
            exps.extend(e)
            coefs.extend(c)
            atom.append(ia)
            n += len(e)
    return dict(center=np.array(center, dtype=np.float64).reshape(-1, 3),
                l=np.array(ls, dtype=np.int32), nprim=np.array(nprim, dtype=np.int32),
                prim_off=np.array(off, dtype=np.int32), exps=np.array(exps, dtype=np.float64),
                coefs=np.array(coefs, dtype=np.float64), atom=np.array(atom, dtype=np.int32))


def nbf(basis: dict) -> int:
    return int(sum(ncart(int(l)) for l in basis["l"]))


def bf_centers(basis: dict) -> np.ndarray:
    """Centre of every Cartesian basis function, [nbf, 3] bohr."""
    rows = []
    for xyz, l in zip(basis["center"], basis["l"]):
        rows += [xyz] * ncart(int(l))
    return np.array(rows).reshape(-1, 3)


def density(basis: dict, seed: int, decay_per_ang=0.3) -> np.ndarray:
    """D_mn = u_mn * exp(-0.3 * r_mn / A) with u ~ U[-1,1] on the upper triangle
    (diagonal included), mirrored to a symmetric matrix."""
    rng = np.random.Generator(np.random.PCG64(20_000 + seed))
    cen = bf_centers(basis) * BOHR_ANGSTROM
    n = cen.shape[0]
    u = rng.uniform(-1.0, 1.0, (n, n))
    u = np.triu(u)
    u = u + np.triu(u, 1).T
    r = np.linalg.norm(cen[:, None, :] - cen[None, :, :], axis=-1)
    return np.ascontiguousarray(u * np.exp(-decay_per_ang * r))


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

CONFIG_NAMES = {
    0: "water trimer, 6-31G(d)-shaped synthetic basis, FP64, tau=1e-12",
    1: "C20H42 zigzag, 6-31G(d)-shaped synthetic basis, FP64, tau=1e-10",
    2: "(H2O)64 liquid-density sphere, 6-31G(d)-shaped synthetic basis, tau=1e-10",
}


def problem(config: int, seed: int = 0, carbons: int = 20, waters: int = 64) -> Problem:
    """The seeded synthetic workload for config 0 (water trimer), 1 (C20H42,
    or another zigzag alkane length via `carbons`) or 2 ((H2O)64 sphere, or
    another cluster size via `waters`: 334 gives the 1,002-atom cluster)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if config == 0:
        mol, tau = water_chain_cluster(3, rng), 1e-12
    elif config == 1:
        mol, tau = alkane_zigzag(carbons), 1e-10
    elif config == 2:
        mol, tau = water_sphere_cluster(waters, rng), 1e-10
    else:
        raise ValueError(f"unknown config {config}")
    basis = make_basis(mol, basis_set("dz", seed))
    D = density(basis, seed)
    name = CONFIG_NAMES[config]
    if config == 1 and carbons != 20:
        name = name.replace("C20H42", f"C{carbons}H{2 * carbons + 2}")
    if config == 2 and waters != 64:
        name = name.replace("(H2O)64", f"(H2O){waters}")
    return Problem(name, mol, basis, D, tau, dict(config=config, seed=seed, carbons=carbons, waters=waters))


def batch_molecules(n: int = 256, seed: int = 0, min_atoms: int = 5, max_atoms: int = 40) -> list:
    """Seeded molecules of uneven size (min_atoms..max_atoms atoms): a water
    cluster (H2O)_m, a zigzag alkane C_kH_(2k+2) with random torsions, or a
    non-overlapping union of one of each."""
    rng = np.random.Generator(np.random.PCG64(30_000 + seed))
    out = []
    while len(out) < n:
        kind = int(rng.integers(0, 3))
        if kind == 0:
            mol = water_chain_cluster(int(rng.integers(2, 14)), rng)
        elif kind == 1:
            k = int(rng.integers(1, 13))
            tors = rng.uniform(-np.pi, np.pi, max(0, k - 3)) if k > 3 else None
            mol = alkane_zigzag(k, torsions=tors)
            if _clash(mol):
                continue
        else:
            k = int(rng.integers(1, 7))
            a = alkane_zigzag(k)
            w = water_chain_cluster(int(rng.integers(2, 6)), rng)
            shift = (a.coords.max(axis=0) - w.coords.min(axis=0)) + np.array([6.0, 0.0, 0.0]) / BOHR_ANGSTROM
            w = Molecule(w.symbols, w.coords + np.array([shift[0], 0.0, 0.0]))
            mol = combine(a, w)
        if min_atoms <= mol.natom <= max_atoms:
            out.append(mol)
    return out


def _clash(mol: Molecule, dmin_ang=0.9) -> bool:
    x = mol.coords * BOHR_ANGSTROM
    d = np.linalg.norm(x[:, None] - x[None], axis=-1)
    np.fill_diagonal(d, 1e9)
    return bool(d.min() < dmin_ang)


def batch_problems(n: int = 256, seed: int = 0, kind: str = "tz", tau: float = 1e-10) -> list:
    """The batched workload: n seeded molecules with the triple-zeta-shaped basis
    up to f and each its own distance-decaying density."""
    table = basis_set(kind, seed)
    probs = []
    for i, mol in enumerate(batch_molecules(n, seed)):
        basis = make_basis(mol, table)
        probs.append(Problem(f"batch molecule {i} ({mol.natom} atoms)", mol, basis, density(basis, 1000 * seed + i),
                             tau, dict(batch_index=i, seed=seed)))
    return probs


def _nonbonded_clash(mol: Molecule, hh_ang=1.5, cc_ang=2.4) -> bool:
    """True if two H atoms are closer than hh_ang or two non-bonded carbons
    (farther than a bond, 1.7 A) closer than cc_ang."""
    x = mol.coords * BOHR_ANGSTROM
    sym = np.array(mol.symbols)
    d = np.linalg.norm(x[:, None] - x[None], axis=-1)
    np.fill_diagonal(d, 1e9)
    h = sym == "H"
    c = sym == "C"
    if h.sum() > 1 and d[np.ix_(h, h)].min() < hh_ang:
        return True
    dc = d[np.ix_(c, c)]
    return bool(((dc > 1.7) & (dc < cc_ang)).any())


def scf_conformations(n: int = 500, seed: int = 0) -> list:
    """Seeded conformations for the SCF / learned-guess workload, alternating
    C8-C16 alkanes (torsions near anti/gauche, +-15 deg, clash-rejected) and
    (H2O)8-16 clusters."""
    rng = np.random.Generator(np.random.PCG64(40_000 + seed))
    out = []
    while len(out) < n:
        if len(out) % 2 == 0:
            k = int(rng.integers(8, 17))
            tors = rng.choice([math.pi, math.pi / 3, -math.pi / 3], k - 3, p=[0.6, 0.2, 0.2])
            tors = tors + rng.normal(0, math.radians(15), k - 3)
            mol = alkane_zigzag(k, torsions=tors)
            if _nonbonded_clash(mol):
                continue
        else:
            mol = water_chain_cluster(int(rng.integers(8, 17)), rng)
        out.append(mol)
    return out


def custom_problem(mol: Molecule, kind="dz", seed=0, tau=1e-10, name="custom") -> Problem:
    basis = make_basis(mol, basis_set(kind, seed))
    return Problem(name, mol, basis, density(basis, seed), tau, dict(seed=seed))


def single_shell_basis(shells, seed=0) -> dict:
    """Basis from an explicit list of (l, center_bohr[3], exps, coefs)."""
    center, ls, nprim, off, exps, coefs, atom = [], [], [], [], [], [], []
    n = 0
    for i, (l, c, e, k) in enumerate(shells):
        center.append(np.asarray(c, float))
        ls.append(l)
        nprim.append(len(e))
        off.append(n)
        exps.extend(e)
        coefs.extend(k)
        atom.append(i)
        n += len(e)
    return dict(center=np.array(center, dtype=np.float64).reshape(-1, 3),
                l=np.array(ls, dtype=np.int32), nprim=np.array(nprim, dtype=np.int32),
                prim_off=np.array(off, dtype=np.int32), exps=np.array(exps, dtype=np.float64),
                coefs=np.array(coefs, dtype=np.float64), atom=np.array(atom, dtype=np.int32))


def random_shells(rng: np.random.Generator, ls, spread=1.5, kmax=3) -> dict:
    """Random shells with the given angular momenta, centres within +-spread bohr."""
    shells = []
    for l in ls:
        K = int(rng.integers(1, kmax + 1))
        a0 = rng.uniform(0.1, 0.3)
        b = rng.uniform(2.5, 4.0)
        e = (a0 * b ** np.arange(K))[::-1].copy()
        c = rng.uniform(0.1, 1.0, K)
        shells.append((l, rng.uniform(-spread, spread, 3), e, c))
    return single_shell_basis(shells)
