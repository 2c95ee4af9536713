"""Density decay bound of the heuristic linear-scaling exchange
(arXiv:2407.21445, Sec. 4.3.1, Eq. density_bound |D_cd| <= H exp(-Lambda |CD|)),
written out plainly for the tests.  Test infrastructure: only tests/,
__graft_entry__.smoke() and bench.py's CPU legs use the oracle.

Readings of the passage (the paper leaves them open):
  - the density elements are binned per pair of shells on different atoms,
    with the shell-block maximum max|D| and the distance of the shell centres;
    bins are 0.5 bohr wide;
  - the least-squares line is fitted to ln(bin maximum) at the bin centres;
    ln H is then raised until the line lies above every bin's maximum over the
    whole bin (its far edge when Lambda > 0), so the bound holds for every
    binned element;
  - R_a = max |AC| over the shells c that a forms a kept (significant) pair
    with -- the printed condition G_[ac] < tau read as G >= tau, since only
    significant pairs enter the bound; G_a the largest Schwarz factor of those
    pairs.  A pair is kept when G_ac * max G >= tau and at least one of its
    primitive pairs survives G_[ac] * max G >= tau * eps_p (Sec. 3.2).
"""
from __future__ import annotations

import math

import numpy as np

BIN = 0.5  # bohr


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def shell_block_max(basis: dict, D: np.ndarray) -> np.ndarray:
    """max |D_mn| over the functions of every pair of shells."""
    off = np.concatenate([[0], np.cumsum([ncart(int(l)) for l in basis["l"]])])
    ns = len(basis["l"])
    out = np.zeros((ns, ns))
    A = np.abs(D)
    for a in range(ns):
        for b in range(ns):
            out[a, b] = A[off[a]:off[a + 1], off[b]:off[b + 1]].max()
    return out


def shell_atoms(basis: dict) -> np.ndarray:
    """Atom index per shell: the description's, else shells sharing a centre."""
    if basis.get("atom") is not None:
        return np.asarray(basis["atom"])
    c = basis["center"]
    out = np.arange(len(c))
    for s in range(len(c)):
        for t in range(s):
            if np.all(c[t] == c[s]):
                out[s] = out[t]
                break
    return out


def centre_distance(c: np.ndarray, a: int, b: int) -> float:
    """|A - B| evaluated left to right, (dx*dx + dy*dy) + dz*dz."""
    dx, dy, dz = c[a, 0] - c[b, 0], c[a, 1] - c[b, 1], c[a, 2] - c[b, 2]
    return math.sqrt((dx * dx + dy * dy) + dz * dz)


def decay_bins(basis: dict, Dsh: np.ndarray) -> dict:
    """{bin index: largest block maximum} over pairs of shells on different atoms."""
    atom = shell_atoms(basis)
    c = basis["center"]
    ns = len(atom)
    bins = {}
    for a in range(ns):
        for b in range(a + 1, ns):
            if atom[a] == atom[b] or not Dsh[a, b] > 0.0:
                continue
            k = int(math.floor(centre_distance(c, a, b) / BIN))
            bins[k] = max(bins.get(k, 0.0), Dsh[a, b])
    return bins


def decay_fit(bins: dict) -> tuple[float, float]:
    """(H, Lambda): least squares of ln max on the bin centres, then ln H
    raised to bound every bin over its whole width."""
    ks = sorted(bins)
    if not ks:
        return 0.0, 0.0
    x = np.array([(k + 0.5) * BIN for k in ks])
    y = np.log(np.array([bins[k] for k in ks]))
    lam = 0.0
    if len(ks) >= 2:
        n = len(ks)
        den = n * np.sum(x * x) - np.sum(x) ** 2
        if den > 0.0:
            lam = -(n * np.sum(x * y) - np.sum(x) * np.sum(y)) / den
    edge = np.array([(k + 1 if lam > 0.0 else k) * BIN for k in ks])
    return float(np.exp(np.max(y + lam * edge))), float(lam)


def kept_pairs(basis: dict, G: np.ndarray, Gp: np.ndarray, tau: float, eps_p: float = 1e-3):
    """Unordered shell pairs (a <= b) the J/K build keeps (Sec. 3.2 pruning)."""
    ns = len(basis["l"])
    npr = basis["nprim"]
    gmax = G.max()
    out = []
    for a in range(ns):
        for b in range(a, ns):
            if G[a, b] * gmax < tau:
                continue
            prims = Gp[a, b, :npr[a] * npr[b]]
            if eps_p > 0.0 and not np.any(prims * gmax >= tau * eps_p):
                continue
            out.append((a, b))
    return out


def shell_radii(basis: dict, G: np.ndarray, Gp: np.ndarray, tau: float, eps_p: float = 1e-3):
    """R_s (largest centre distance to a kept partner) and G_s (largest
    Schwarz factor of its kept pairs)."""
    ns = len(basis["l"])
    c = basis["center"]
    R = np.zeros(ns)
    Gs = np.zeros(ns)
    for a, b in kept_pairs(basis, G, Gp, tau, eps_p):
        d = float(np.linalg.norm(c[a] - c[b]))
        R[a] = max(R[a], d)
        R[b] = max(R[b], d)
        Gs[a] = max(Gs[a], G[a, b])
        Gs[b] = max(Gs[b], G[a, b])
    return R, Gs
