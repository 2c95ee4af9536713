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

import itertools
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


_TERMS = {}


def _rep_terms(l: int):
    """Expansion of rep_matrix(l, R) as a sum over index tuples: M[g, e] is
    the sum over (i_1..i_l) of c * prod_k R[i_k, j_k]; returned as index arrays
    I, J [T, l] and the scatter matrix S [T, nc*nc] holding the factors c."""
    if l not in _TERMS:
        comps = cart_list(l)
        idx = {c: i for i, c in enumerate(comps)}
        nc = len(comps)
        I, J, rows = [], [], []
        for g, cg in enumerate(comps):
            js = [0] * cg[0] + [1] * cg[1] + [2] * cg[2]
            for it in itertools.product(range(3), repeat=l):
                e = (it.count(0), it.count(1), it.count(2))
                I.append(list(it))
                J.append(js)
                rows.append((g * nc + idx[e], _cnorm(cg) / _cnorm(e)))
        S = np.zeros((len(rows), nc * nc))
        for t, (k, c) in enumerate(rows):
            S[t, k] = c
        _TERMS[l] = (np.array(I, dtype=np.int64).reshape(len(rows), l), np.array(J, dtype=np.int64).reshape(len(rows), l), S)
    return _TERMS[l]


def rep_matrices(l: int, Rs: np.ndarray) -> np.ndarray:
    """rep_matrix(l, R) for a stack of rotations Rs [B, 3, 3] -> [B, nc, nc]."""
    nc = (l + 1) * (l + 2) // 2
    B = Rs.shape[0]
    if l == 0:
        return np.ones((B, 1, 1))
    I, J, S = _rep_terms(l)
    prod = np.prod(Rs[:, I, J], axis=2)
    return (prod @ S).reshape(B, nc, nc)


def _atom_M_stack(ls, reps):
    """Block-diagonal atom matrices [B, n, n] from per-l matrices reps[l] [B, ., .]."""
    B = next(iter(reps.values())).shape[0]
    n = sum((l + 1) * (l + 2) // 2 for l in ls)
    M = np.zeros((B, n, n))
    o = 0
    for l in ls:
        k = (l + 1) * (l + 2) // 2
        M[:, o:o + k, o:o + k] = reps[l]
        o += k
    return M


def _pair_groups(sh, pairs):
    """Pairs grouped by the shell lists of their two atoms."""
    groups = {}
    for k, (a, b) in enumerate(pairs):
        groups.setdefault((tuple(sh[a]["ls"]), tuple(sh[b]["ls"])), []).append(k)
    return {key: np.array(v, dtype=np.int64) for key, v in groups.items()}


def _block_index(sh, pairs, ps, na, nb):
    fa = np.array([sh[pairs[k][0]]["first"] for k in ps])
    fb = np.array([sh[pairs[k][1]]["first"] for k in ps])
    rows = fa[:, None] + np.arange(na)[None, :]
    cols = fb[:, None] + np.arange(nb)[None, :]
    return rows, cols


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
    with their rotation (rows ex, ey, ez) and feature vectors.

    Frame: for a != b, ez along A -> B and the nearest other atom to the
    pair's midpoint fixes ex; for a == b (the atom's own block) ez points to
    the nearest other atom and the second nearest fixes ex.  Features:
    elements of a and b (one-hot), a == b, |AB|/5, radial basis exp(-(|AB| -
    r_k)^2), and for the NNB nearest other atoms their local coordinates / 5,
    1 / (1 + distance) and element (one-hot); neighbours ordered by distance
    to the midpoint, ties by index."""
    X = np.asarray(mol.coords, dtype=np.float64)
    el = np.array([ELEM[s] for s in mol.symbols])
    n = len(el)
    D = np.linalg.norm(X[:, None] - X[None], axis=-1)
    key = el * (n + 1) + np.arange(n)  # (element, index) order
    keep = ((key[:, None] < key[None, :]) | np.eye(n, dtype=bool)) & (D <= PAIR_CUTOFF)
    A, B = np.nonzero(keep)  # row-major: a ascending, then b
    P = len(A)
    if P == 0:
        return [], [], np.zeros((0, NFEAT), dtype=np.float32)
    mid = 0.5 * (X[A] + X[B])
    dm = np.linalg.norm(X[None, :, :] - mid[:, None, :], axis=-1)
    dm[np.arange(P), A] = np.inf
    dm[np.arange(P), B] = np.inf
    order = np.argsort(dm, axis=1, kind="stable")
    nothers = np.where(A == B, n - 1, n - 2)
    self_pair = A == B
    z3 = np.array([0.0, 0.0, 1.0])
    x3 = np.array([1.0, 0.0, 0.0])
    o0 = order[:, 0] if n > 0 else np.zeros(P, dtype=np.int64)
    o1 = order[:, 1] if n > 1 else np.zeros(P, dtype=np.int64)
    ez = np.where(self_pair[:, None], np.where((nothers > 0)[:, None], X[o0] - X[A], z3), X[B] - X[A])
    ref = np.where(self_pair[:, None], np.where((nothers > 1)[:, None], X[o1] - X[A], x3),
                   np.where((nothers > 0)[:, None], X[o0] - mid, z3))
    ez = ez / np.linalg.norm(ez, axis=1, keepdims=True)
    v = ref - np.sum(ref * ez, axis=1, keepdims=True) * ez
    bad = np.linalg.norm(v, axis=1) < 1e-6
    if bad.any():
        tmp = np.where((np.abs(ez[:, 0]) < 0.9)[:, None], x3, np.array([0.0, 1.0, 0.0]))
        v2 = tmp - np.sum(tmp * ez, axis=1, keepdims=True) * ez
        v = np.where(bad[:, None], v2, v)
    ex = v / np.linalg.norm(v, axis=1, keepdims=True)
    ey = np.cross(ez, ex)
    R = np.stack([ex, ey, ez], axis=1)  # [P, 3, 3], rows ex, ey, ez
    f = np.zeros((P, NFEAT), dtype=np.float32)
    f[np.arange(P), el[A]] = 1.0
    f[np.arange(P), 3 + el[B]] = 1.0
    f[:, 6] = self_pair
    dab = D[A, B]
    f[:, 7] = dab / 5.0
    f[:, 8:8 + len(RBF)] = np.exp(-((dab[:, None] - RBF[None, :]) ** 2))
    o = 8 + len(RBF)
    for k in range(min(NNB, max(n - 1, 0))):
        c = order[:, k]
        valid = k < nothers
        loc = np.einsum("pij,pj->pi", R, X[c] - mid)
        blk = np.zeros((P, 7), dtype=np.float64)
        blk[:, 0:3] = loc / 5.0
        blk[:, 3] = 1.0 / (1.0 + np.linalg.norm(loc, axis=1))
        blk[np.arange(P), 4 + el[c]] = 1.0
        f[valid, o + 7 * k:o + 7 * k + 7] = blk[valid]
    pairs = list(zip(A.tolist(), B.tolist()))
    return pairs, list(R), f


def _reps(sh, pairs, frames, transpose=False):
    Rs = np.array(frames).reshape(-1, 3, 3)
    if transpose:
        Rs = np.transpose(Rs, (0, 2, 1))
    ls = sorted({l for a in sh.values() for l in a["ls"]})
    return {l: rep_matrices(l, Rs) for l in ls}


def blocks_to_local(D: np.ndarray, mol, basis, pairs, frames):
    """Targets: each pair block of D in its local frame (Ma^T D_ab Mb with M
    the Cartesian representation of the frame), padded to 15 x 15, with the
    mask of its valid entries."""
    sh = atom_shells(basis)
    T = np.zeros((len(pairs), NOUT), dtype=np.float32)
    Mk = np.zeros((len(pairs), NOUT), dtype=np.float32)
    if not pairs:
        return T, Mk
    reps = _reps(sh, pairs, frames)
    for (lsa, lsb), ps in _pair_groups(sh, pairs).items():
        sub = {l: r[ps] for l, r in reps.items()}
        Ma, Mb = _atom_M_stack(lsa, sub), _atom_M_stack(lsb, sub)
        na, nb = Ma.shape[1], Mb.shape[1]
        rows, cols = _block_index(sh, pairs, ps, na, nb)
        blk = D[rows[:, :, None], cols[:, None, :]]
        loc = np.transpose(Ma, (0, 2, 1)) @ blk @ Mb
        t = np.zeros((len(ps), MAXB, MAXB))
        t[:, :na, :nb] = loc
        m = np.zeros((len(ps), MAXB, MAXB))
        m[:, :na, :nb] = 1.0
        T[ps] = t.reshape(len(ps), NOUT)
        Mk[ps] = m.reshape(len(ps), NOUT)
    return T, Mk


def local_to_density(Y: np.ndarray, mol, basis, pairs, frames, nbf: int) -> np.ndarray:
    """Predicted local blocks back to the global basis: Ma^-T Y_ab Mb^-1, with
    M(R)^-1 = M(R^T) (the Cartesian functions carry a representation of the
    rotation group); own-atom blocks symmetrised."""
    sh = atom_shells(basis)
    D = np.zeros((nbf, nbf))
    if not pairs:
        return D
    inv = _reps(sh, pairs, frames, transpose=True)
    A = np.array([p[0] for p in pairs])
    Bv = np.array([p[1] for p in pairs])
    for (lsa, lsb), ps in _pair_groups(sh, pairs).items():
        sub = {l: r[ps] for l, r in inv.items()}
        Ia, Ib = _atom_M_stack(lsa, sub), _atom_M_stack(lsb, sub)
        na, nb = Ia.shape[1], Ib.shape[1]
        loc = Y[ps].reshape(len(ps), MAXB, MAXB)[:, :na, :nb].astype(np.float64)
        same = A[ps] == Bv[ps]
        if same.any():
            loc[same] = 0.5 * (loc[same] + np.transpose(loc[same], (0, 2, 1)))
        blk = np.transpose(Ia, (0, 2, 1)) @ loc @ Ib
        rows, cols = _block_index(sh, pairs, ps, na, nb)
        D[rows[:, :, None], cols[:, None, :]] = blk
        off = ~same
        if off.any():
            D[cols[off][:, :, None], rows[off][:, None, :]] = np.transpose(blk[off], (0, 2, 1))
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
