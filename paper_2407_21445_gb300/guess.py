"""Learned initial density for the RHF driver: an atom-pair MLP (the library's
fock_mlp kernels) predicts, for every atom pair, the correction from the
superposition-of-atomic-densities (SAD) block to the converged density block
in a local frame of the pair; the blocks are rotated back, added to the SAD
density and projected onto an idempotent density (natural orbitals of D S,
the nocc largest kept).

Host-side input preparation only (frames, features, block rotations); the
network's forward and backward passes run in the library's CUDA kernels.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .fock import MLP

ELEM = {"H": 0, "C": 1, "O": 2}
MAXB = 15           # functions per atom in the 6-31G(d)-shaped basis (heavy atoms)
NOUT = MAXB * MAXB  # flattened block
NNB = 12            # neighbours described in the pair frame
RBF = np.arange(0.0, 12.0, 1.0)
NFEAT = 3 + 3 + 1 + 1 + len(RBF) + NNB * 7
PAIR_CUTOFF = 10.0  # bohr; farther blocks are predicted as zero


def cart_list(l):
    return [(x, y, l - x - y) for x in range(l, -1, -1) for y in range(l - x, -1, -1)]


def _dfact(n):
    return math.prod(range(n, 0, -2)) if n > 0 else 1


def _cnorm(c):
    return 1.0 / math.sqrt(_dfact(2 * c[0] - 1) * _dfact(2 * c[1] - 1) * _dfact(2 * c[2] - 1))


def rep_matrix(l: int, R: np.ndarray) -> np.ndarray:
    """M with phi_global = M phi_local for the normalised Cartesian functions of
    angular momentum l, local coordinates r' = R r (so r = R^T r')."""
    comps = cart_list(l)
    idx = {c: i for i, c in enumerate(comps)}
    M = np.zeros((len(comps), len(comps)))
    for g, cg in enumerate(comps):
        axes = [0] * cg[0] + [1] * cg[1] + [2] * cg[2]  # global factors x_j
        terms = {(0, 0, 0): 1.0}
        for j in axes:  # x_j = sum_i R_ij x'_i
            nt = {}
            for e, w in terms.items():
                for i in range(3):
                    e2 = list(e)
                    e2[i] += 1
                    e2 = tuple(e2)
                    nt[e2] = nt.get(e2, 0.0) + w * R[i, j]
            terms = nt
        for e, w in terms.items():
            M[g, idx[e]] += _cnorm(cg) * w / _cnorm(e)
    return M


def atom_shells(basis: dict):
    """Per atom: list of angular momenta of its shells and its first function."""
    offs = np.concatenate([[0], np.cumsum([(int(l) + 1) * (int(l) + 2) // 2 for l in basis["l"]])])
    out = {}
    for s, (a, l) in enumerate(zip(basis["atom"], basis["l"])):
        out.setdefault(int(a), {"ls": [], "first": int(offs[s])})
        out[int(a)]["ls"].append(int(l))
    return out


def atom_M(ls, R):
    blocks = [rep_matrix(l, R) for l in ls]
    n = sum(b.shape[0] for b in blocks)
    M = np.zeros((n, n))
    o = 0
    for b in blocks:
        k = b.shape[0]
        M[o:o + k, o:o + k] = b
        o += k
    return M


def _frame(ez, ref):
    ez = ez / np.linalg.norm(ez)
    v = ref - np.dot(ref, ez) * ez
    if np.linalg.norm(v) < 1e-6:
        tmp = np.array([1.0, 0.0, 0.0]) if abs(ez[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        v = tmp - np.dot(tmp, ez) * ez
    ex = v / np.linalg.norm(v)
    ey = np.cross(ez, ex)
    return np.stack([ex, ey, ez])


def pair_frames(mol):
    """All atom pairs (a, b), a <= b by (element, index), within PAIR_CUTOFF,
    with their rotation (rows ex, ey, ez) and feature vectors."""
    X = mol.coords
    el = np.array([ELEM[s] for s in mol.symbols])
    n = len(el)
    D = np.linalg.norm(X[:, None] - X[None], axis=-1)
    pairs, frames, feats = [], [], []
    for a in range(n):
        for b in range(n):
            if a != b and (el[a], a) > (el[b], b):
                continue
            if D[a, b] > PAIR_CUTOFF:
                continue
            mid = 0.5 * (X[a] + X[b])
            others = [c for c in range(n) if c != a and c != b]
            dm = np.linalg.norm(X[others] - mid, axis=1) if others else np.zeros(0)
            order = [others[i] for i in np.argsort(dm, kind="stable")]
            if a != b:
                ez = X[b] - X[a]
                ref = X[order[0]] - mid if order else np.array([0.0, 0.0, 1.0])
            else:
                ez = X[order[0]] - X[a] if order else np.array([0.0, 0.0, 1.0])
                ref = X[order[1]] - X[a] if len(order) > 1 else np.array([1.0, 0.0, 0.0])
            R = _frame(ez, ref)
            f = np.zeros(NFEAT, dtype=np.float32)
            f[el[a]] = 1.0
            f[3 + el[b]] = 1.0
            f[6] = 1.0 if a == b else 0.0
            f[7] = D[a, b] / 5.0
            f[8:8 + len(RBF)] = np.exp(-((D[a, b] - RBF) ** 2))
            o = 8 + len(RBF)
            for k, c in enumerate(order[:NNB]):
                loc = R @ (X[c] - mid)
                f[o + 7 * k:o + 7 * k + 3] = loc / 5.0
                f[o + 7 * k + 3] = 1.0 / (1.0 + np.linalg.norm(loc))
                f[o + 7 * k + 4 + el[c]] = 1.0
            pairs.append((a, b))
            frames.append(R)
            feats.append(f)
    return pairs, frames, np.array(feats, dtype=np.float32).reshape(-1, NFEAT)


def blocks_to_local(D: np.ndarray, mol, basis, pairs, frames):
    """Targets: each pair block of D in its local frame, padded to 15 x 15,
    with the mask of its valid entries."""
    sh = atom_shells(basis)
    T = np.zeros((len(pairs), NOUT), dtype=np.float32)
    Mk = np.zeros((len(pairs), NOUT), dtype=np.float32)
    for k, ((a, b), R) in enumerate(zip(pairs, frames)):
        Ma, Mb = atom_M(sh[a]["ls"], R), atom_M(sh[b]["ls"], R)
        na, nb = Ma.shape[0], Mb.shape[0]
        blk = D[sh[a]["first"]:sh[a]["first"] + na, sh[b]["first"]:sh[b]["first"] + nb]
        loc = Ma.T @ blk @ Mb
        t = np.zeros((MAXB, MAXB))
        t[:na, :nb] = loc
        m = np.zeros((MAXB, MAXB))
        m[:na, :nb] = 1.0
        T[k] = t.ravel()
        Mk[k] = m.ravel()
    return T, Mk


def local_to_density(Y: np.ndarray, mol, basis, pairs, frames, nbf: int) -> np.ndarray:
    sh = atom_shells(basis)
    D = np.zeros((nbf, nbf))
    for k, ((a, b), R) in enumerate(zip(pairs, frames)):
        Ma, Mb = atom_M(sh[a]["ls"], R), atom_M(sh[b]["ls"], R)
        na, nb = Ma.shape[0], Mb.shape[0]
        loc = Y[k].reshape(MAXB, MAXB)[:na, :nb].astype(np.float64)
        if a == b:
            loc = 0.5 * (loc + loc.T)
        blk = np.linalg.solve(Ma.T, np.linalg.solve(Mb.T, loc.T).T)  # Ma^-T loc Mb^-1
        fa, fb = sh[a]["first"], sh[b]["first"]
        D[fa:fa + na, fb:fb + nb] = blk
        if a != b:
            D[fb:fb + nb, fa:fa + na] = blk.T
    return D


def project_idempotent(D: torch.Tensor, S: torch.Tensor, X: torch.Tensor, nocc: int) -> torch.Tensor:
    """Closest closed-shell density: the nocc natural orbitals of largest
    occupation of D (in the orthonormal basis X) doubly occupied."""
    Do = X.T @ S @ D @ S @ X
    Do = 0.5 * (Do + Do.T)
    w, V = torch.linalg.eigh(Do)
    C = X @ V[:, -nocc:]
    return 2.0 * C @ C.T


class LearnedGuess:
    """Feature normalisation + the library MLP + density assembly."""

    def __init__(self, hidden: int = 128, max_batch: int = 8192, seed: int = 0):
        self.net = MLP(NFEAT, hidden, NOUT, max_batch, seed)
        self.mu = np.zeros(NFEAT, dtype=np.float32)
        self.sd = np.ones(NFEAT, dtype=np.float32)
        self.max_batch = max_batch

    @classmethod
    def load(cls, path: str, hidden: int = 128, max_batch: int = 8192):
        """A trained network saved by train_guess (parameters and feature
        normaliser)."""
        z = np.load(path)
        g = cls(hidden=hidden, max_batch=max_batch)
        g.net.set_params(z["params"])
        g.mu, g.sd = z["mu"].astype(np.float32), z["sd"].astype(np.float32)
        return g

    def fit_normaliser(self, feats: np.ndarray):
        self.mu = feats.mean(0).astype(np.float32)
        self.sd = (feats.std(0) + 1e-3).astype(np.float32)

    def features(self, feats: np.ndarray) -> np.ndarray:
        return ((feats - self.mu) / self.sd).astype(np.float32)

    def train(self, feats, targets, masks, epochs=60, batch=4096, lr=2e-3, seed=0, log=None):
        dev = "cuda"
        Xa = torch.tensor(self.features(feats), device=dev)
        Ta = torch.tensor(targets, device=dev)
        Ma = torch.tensor(masks, device=dev)
        n = Xa.shape[0]
        g = torch.Generator(device="cpu").manual_seed(seed)
        steps = 0
        hist = []
        total = epochs * ((n + batch - 1) // batch)
        for ep in range(epochs):
            perm = torch.randperm(n, generator=g).to(dev)
            tot = 0.0
            for i in range(0, n, batch):
                idx = perm[i:i + batch]
                X, T, M = Xa[idx].contiguous(), Ta[idx].contiguous(), Ma[idx].contiguous()
                lr_t = lr * 0.5 * (1 + math.cos(math.pi * steps / total))  # cosine schedule
                tot += self.net.loss_backward(X, T, M, norm=float(M.sum())) * len(idx)
                self.net.step(lr=lr_t, weight_decay=1e-6)
                steps += 1
            hist.append(tot / n)
            if log:
                log(f"epoch {ep} loss {tot / n:.3e}")
        return hist

    def predict_local(self, feats: np.ndarray) -> np.ndarray:
        X = torch.tensor(self.features(feats), device="cuda")
        out = []
        for i in range(0, X.shape[0], self.max_batch):
            out.append(self.net.forward(X[i:i + self.max_batch].contiguous()).cpu().numpy())
        return np.concatenate(out) if out else np.zeros((0, NOUT), dtype=np.float32)

    def guess(self, mol, basis, rhf, D_sad: np.ndarray) -> torch.Tensor:
        """SAD density plus the predicted correction, projected to an
        idempotent closed-shell density."""
        pairs, frames, feats = pair_frames(mol)
        Y = self.predict_local(feats)
        D = D_sad + local_to_density(Y, mol, basis, pairs, frames, rhf.S.shape[0])
        Dt = torch.tensor(D, device=rhf.S.device, dtype=rhf.S.dtype)
        return project_idempotent(Dt, rhf.S, rhf.X, rhf.nocc)
