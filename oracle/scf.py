"""Plain CPU closed-shell RHF on the oracle's integrals (test infrastructure
only: the GPU SCF driver is checked against it, nothing else uses it).

Sec. 2.2 of arXiv:2407.21445: the Fock matrix F = h + J - K/2 with
h = T + V, the density D = 2 C_occ C_occ^T, and the Roothaan equations
F C = S C eps, iterated to self-consistency.  The energy is
E = 1/2 tr(D (h + F)) + E_nuc.  Orthogonalisation is canonical, dropping
overlap eigenvalues below 1e-7 (the synthetic bases can be nearly linearly
dependent); convergence is accelerated by Pulay's DIIS on the commutator
X^T (F D S - S D F) X.  Nothing here is shared with the GPU package.
"""
from __future__ import annotations

import numpy as np

from . import jk, kinetic, nuclear, overlap


def nuclear_repulsion(Z, xyz) -> float:
    """E_nuc = sum_{i<j} Z_i Z_j / |R_i - R_j| (bohr)."""
    Z = np.asarray(Z, dtype=np.float64)
    xyz = np.asarray(xyz, dtype=np.float64)
    e = 0.0
    for i in range(len(Z)):
        for j in range(i):
            e += Z[i] * Z[j] / np.linalg.norm(xyz[i] - xyz[j])
    return e


def rhf(basis: dict, Z, xyz, nocc: int, tau: float = 0.0, D0=None, iters: int = 200,
        conv_e: float = 1e-10, conv_comm: float = 1e-7, ndiis: int = 8) -> dict:
    """Converged closed-shell RHF: {"energy", "electronic", "eps", "D",
    "iterations"}; D0 the initial density (None: the core Hamiltonian's).
    Raises if it does not converge within `iters` iterations."""
    S = overlap(basis)
    h = kinetic(basis) + nuclear(basis, Z, xyz)
    s, U = np.linalg.eigh(S)
    keep = s > 1e-7
    X = U[:, keep] / np.sqrt(s[keep])
    enuc = nuclear_repulsion(Z, xyz)

    def density(F):
        eps, C = np.linalg.eigh(X.T @ F @ X)
        C = X @ C
        return eps, 2.0 * C[:, :nocc] @ C[:, :nocc].T

    D = density(h)[1] if D0 is None else np.asarray(D0, dtype=np.float64)
    Fs, Es = [], []
    e_prev = None
    for it in range(iters):
        J, K = jk(basis, D, tau)
        F = h + J - 0.5 * K
        e_el = 0.5 * float(np.sum(D * (h + F)))
        err = X.T @ (F @ D @ S - S @ D @ F) @ X
        if e_prev is not None and abs(e_el - e_prev) < conv_e and np.abs(err).max() < conv_comm:
            eps, _ = density(F)
            return {"energy": e_el + enuc, "electronic": e_el, "eps": eps, "D": D, "iterations": it}
        e_prev = e_el
        Fs.append(F)
        Es.append(err)
        Fs, Es = Fs[-ndiis:], Es[-ndiis:]
        n = len(Fs)
        Fx = F
        if n >= 2:
            B = -np.ones((n + 1, n + 1))
            B[n, n] = 0.0
            for i in range(n):
                for j in range(n):
                    B[i, j] = np.sum(Es[i] * Es[j])
            rhs = np.zeros(n + 1)
            rhs[n] = -1.0
            c = np.linalg.lstsq(B, rhs, rcond=None)[0]  # singular when the errors vanish
            Fx = sum(c[i] * Fs[i] for i in range(n))
        D = density(Fx)[1]
    raise RuntimeError("oracle RHF did not converge")
