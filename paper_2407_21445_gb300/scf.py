"""Restricted Hartree-Fock driver on the GPU (Sec. 2.2: FC = SCe,
F = h + J - K/2, D = 2 C_occ C_occ^T).

J and K come from libfock.so; the one-electron integrals from
fock_one_electron; the small dense linear algebra (canonical
orthogonalisation, DIIS, FP64 eigendecomposition) uses torch.linalg on the
GPU.  Initial guesses: superposition of atomic densities (SAD) or a density
supplied by the caller (the learned guess of guess.py).

Incremental Fock build (the paper names it as future work in Sec. 7 and notes
in Sec. 6.1 that it was switched off in the codes it compares with): J and K
are linear in D, so J(D_n) = J(D_m) + J(D_n - D_m).  With incremental=True
every iteration builds J and K of the density change since the last build and
adds them; the density-weighted screening of the library then weighs each
quartet by |D_n - D_m|, which shrinks as the SCF converges, so ever fewer
quartets are evaluated.  A full build every `rebuild_every` iterations
bounds the accumulation of screening errors.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from .fock import FOCK_FP64, JKBuilder, fock_one_electron, make_opts


def nuclear_repulsion(Z, xyz) -> float:
    Z = np.asarray(Z, dtype=np.float64)
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    e = 0.0
    for i in range(len(Z)):
        d = np.linalg.norm(xyz[i + 1:] - xyz[i], axis=1)
        e += float(np.sum(Z[i] * Z[i + 1:] / d))
    return e


@dataclass
class SCFResult:
    energy: float
    D: torch.Tensor
    iterations: int
    converged: bool
    energies: list


class RHF:
    """Closed-shell RHF for one molecule (Z, xyz in bohr) in a given basis."""

    def __init__(self, Z, xyz, basis: dict, tau: float = 1e-10, opts=None, lindep: float = 1e-7,
                 charge: int = 0, incremental: bool = False, rebuild_every: int = 8):
        self.Z = np.asarray(Z, dtype=np.float64)
        self.xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
        self.basis = basis
        self.tau = tau
        self.builder = JKBuilder(basis, tau, opts if opts is not None else make_opts(FOCK_FP64))
        S, T, V = fock_one_electron(basis, self.Z, self.xyz)
        self.S, self.h = S, T + V
        self.enuc = nuclear_repulsion(self.Z, self.xyz)
        nel = int(round(self.Z.sum())) - charge
        if nel % 2:
            raise ValueError("closed-shell RHF needs an even electron count")
        self.nocc = nel // 2
        s, U = torch.linalg.eigh(S)
        keep = s > lindep  # canonical orthogonalisation (near-linear dependence)
        self.X = U[:, keep] / torch.sqrt(s[keep])
        self.incremental = bool(incremental)
        self.rebuild_every = max(1, int(rebuild_every))
        self._ref = None        # (D_m, J(D_m), K(D_m)) of the last build
        self._since_full = 0
        self.build_densities = []  # the density each J/K build was given (for statistics)

    def density_from_fock(self, F: torch.Tensor, nocc=None, occ=None) -> torch.Tensor:
        Fo = self.X.T @ F @ self.X
        e, Co = torch.linalg.eigh(Fo)
        C = self.X @ Co
        if occ is None:
            Cocc = C[:, : (self.nocc if nocc is None else nocc)]
            return 2.0 * Cocc @ Cocc.T
        w = torch.as_tensor(occ, dtype=C.dtype, device=C.device)
        Cn = C[:, : len(occ)]
        return (Cn * w) @ Cn.T

    def core_guess(self) -> torch.Tensor:
        return self.density_from_fock(self.h)

    def fock(self, D):
        if not self.incremental:
            J, K = self.builder.build(D)
            self.build_densities.append(("full", D))
            return self.h + J - 0.5 * K
        if self._ref is None or self._since_full >= self.rebuild_every:
            J, K = self.builder.build(D)
            self._since_full = 0
            self.build_densities.append(("full", D))
        else:
            dD = D - self._ref[0]
            dJ, dK = self.builder.build(dD)
            J, K = self._ref[1] + dJ, self._ref[2] + dK
            self._since_full += 1
            self.build_densities.append(("delta", dD))
        self._ref = (D.clone(), J, K)
        return self.h + J - 0.5 * K

    def energy(self, D, F) -> float:
        return float(0.5 * torch.sum(D * (self.h + F))) + self.enuc

    def run(self, D0: torch.Tensor, max_iter: int = 128, e_conv: float = 1e-8, err_conv: float = 1e-6,
            diis_size: int = 8) -> SCFResult:
        """Pulay DIIS iterations from D0; converged when |dE| < e_conv and the
        orthogonalised commutator FDS - SDF is below err_conv (max abs)."""
        D = D0
        focks, errs, energies = [], [], []
        e_prev = None
        for it in range(1, max_iter + 1):
            F = self.fock(D)
            E = self.energy(D, F)
            energies.append(E)
            FDS = F @ D @ self.S
            err = self.X.T @ (FDS - FDS.T) @ self.X
            emax = float(err.abs().max())
            if e_prev is not None and abs(E - e_prev) < e_conv and emax < err_conv:
                return SCFResult(E, D, it, True, energies)
            e_prev = E
            focks.append(F)
            errs.append(err)
            if len(focks) > diis_size:
                focks.pop(0)
                errs.pop(0)
            Fx = F
            n = len(focks)
            if n >= 2:
                B = torch.empty((n + 1, n + 1), dtype=F.dtype, device=F.device)
                for i in range(n):
                    for j in range(i, n):
                        B[i, j] = B[j, i] = torch.sum(errs[i] * errs[j])
                B[n, :] = -1.0
                B[:, n] = -1.0
                B[n, n] = 0.0
                rhs = torch.zeros(n + 1, dtype=F.dtype, device=F.device)
                rhs[n] = -1.0
                try:
                    c = torch.linalg.solve(B, rhs)
                    Fx = sum(c[i] * focks[i] for i in range(n))
                except RuntimeError:
                    Fx = F
            D = self.density_from_fock(Fx)
        return SCFResult(energies[-1], D, max_iter, False, energies)


# --------------------------------------------------------------------------
# superposition of atomic densities
# --------------------------------------------------------------------------

_SAD_CACHE: dict = {}


def atomic_density(symbol: str, Zval: int, shells, tau: float = 1e-12, iters: int = 60) -> np.ndarray:
    """Spherically averaged density of one atom: fractional-occupation SCF in
    the atom's own basis (electrons of a partly filled degenerate level are
    spread evenly over it)."""
    import molgen
    key = (symbol, tuple((l, tuple(e), tuple(c)) for l, e, c in shells))
    if key in _SAD_CACHE:
        return _SAD_CACHE[key]
    bas = molgen.single_shell_basis([(l, [0.0, 0.0, 0.0], e, c) for l, e, c in shells])
    n = int(sum((l + 1) * (l + 2) // 2 for l in bas["l"]))
    Zs = [float(Zval)]
    xyz = [[0.0, 0.0, 0.0]]
    S, T, V = fock_one_electron(bas, Zs, xyz)
    h = T + V
    builder = JKBuilder(bas, tau)
    s, U = torch.linalg.eigh(S)
    keep = s > 1e-7
    X = U[:, keep] / torch.sqrt(s[keep])

    def dens(F):
        e, Co = torch.linalg.eigh(X.T @ F @ X)
        C = X @ Co
        e = e.cpu().numpy()
        occ = np.zeros(len(e))
        left = float(Zval)
        i = 0
        while left > 1e-12 and i < len(e):
            j = i
            while j + 1 < len(e) and abs(e[j + 1] - e[i]) < 1e-3 * max(1.0, abs(e[i])):
                j += 1
            cap = 2.0 * (j - i + 1)
            put = min(cap, left)
            occ[i:j + 1] = put / (j - i + 1)
            left -= put
            i = j + 1
        w = torch.tensor(occ, dtype=C.dtype, device=C.device)
        return (C * w) @ C.T

    D = dens(h)
    for _ in range(iters):
        J, K = builder.build(D)
        Dn = dens(h + J - 0.5 * K)
        if float((Dn - D).abs().max()) < 1e-9:
            D = Dn
            break
        D = 0.5 * D + 0.5 * Dn
    out = D.cpu().numpy()
    _SAD_CACHE[key] = out
    builder.close()
    return out


def sad_guess(mol, table: dict, device="cuda") -> torch.Tensor:
    """Block-diagonal superposition of the atoms' spherically averaged densities."""
    blocks = []
    for sym, Zv in zip(mol.symbols, mol.Z):
        blocks.append(atomic_density(sym, int(Zv), table[sym]))
    n = sum(b.shape[0] for b in blocks)
    D = np.zeros((n, n))
    o = 0
    for b in blocks:
        k = b.shape[0]
        D[o:o + k, o:o + k] = b
        o += k
    return torch.tensor(D, device=device)
