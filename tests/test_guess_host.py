"""Host-side pieces of the learned guess (no GPU): Cartesian rotation
representations and the local-frame block round trip."""
import numpy as np

import molgen
from paper_2407_21445_gb300 import guess


def test_rep_matrix_is_a_representation(rng):
    for l in (0, 1, 2, 3):
        R1 = molgen.random_rotation(rng)
        R2 = molgen.random_rotation(rng)
        M12 = guess.rep_matrix(l, R1 @ R2)
        # phi_global = M(R) phi_local with r' = R r; composing rotations
        assert np.allclose(guess.rep_matrix(l, R2) @ guess.rep_matrix(l, R1), M12, atol=1e-12) or \
            np.allclose(guess.rep_matrix(l, R1) @ guess.rep_matrix(l, R2), M12, atol=1e-12)
        assert np.allclose(guess.rep_matrix(l, R1) @ guess.rep_matrix(l, R1.T), np.eye(len(guess.cart_list(l))),
                           atol=1e-12)
    R = molgen.random_rotation(rng)
    assert np.allclose(guess.rep_matrix(1, R), R.T, atol=1e-14)


def test_local_frame_round_trip(rng):
    mol = molgen.water_chain_cluster(3, rng)
    bas = molgen.make_basis(mol, molgen.basis_set("dz", 0))
    n = molgen.nbf(bas)
    D = rng.uniform(-1, 1, (n, n))
    D = D + D.T
    pairs, frames, feats = guess.pair_frames(mol)
    assert feats.shape == (len(pairs), guess.NFEAT)
    T, M = guess.blocks_to_local(D, mol, bas, pairs, frames)
    D2 = guess.local_to_density(T, mol, bas, pairs, frames, n)
    # blocks of atom pairs beyond the cutoff are not predicted
    sh = guess.atom_shells(bas)
    near = np.zeros((n, n), dtype=bool)
    for a, b in pairs:
        fa, fb = sh[a]["first"], sh[b]["first"]
        na = sum((l + 1) * (l + 2) // 2 for l in sh[a]["ls"])
        nb = sum((l + 1) * (l + 2) // 2 for l in sh[b]["ls"])
        near[fa:fa + na, fb:fb + nb] = near[fb:fb + nb, fa:fa + na] = True
    assert near.any()
    assert np.abs(D2 - D)[near].max() < 1e-5  # targets are float32
    assert np.abs(D2)[~near].max() == 0.0


def test_features_are_rotation_invariant(rng):
    # a jittered geometry: exact distance ties (symmetric structures) make the
    # neighbour order, hence the frame, ambiguous
    base = molgen.alkane_zigzag(3)
    mol = molgen.Molecule(base.symbols, base.coords + rng.normal(0, 0.05, base.coords.shape))
    R = molgen.random_rotation(rng)
    mol2 = molgen.Molecule(mol.symbols, mol.coords @ R.T + rng.uniform(-3, 3, 3))
    _, _, f1 = guess.pair_frames(mol)
    _, _, f2 = guess.pair_frames(mol2)
    assert np.abs(f1 - f2).max() < 1e-4


# ---------------------------------------------------------------------------
# The feature and block definitions written out one atom pair at a time (the
# vectorised code in guess.py must reproduce them: the shipped network was
# trained on these features).

def _ref_frame(ez, ref):
    ez = ez / np.linalg.norm(ez)
    v = ref - np.dot(ref, ez) * ez
    if np.linalg.norm(v) < 1e-6:
        tmp = np.array([1.0, 0.0, 0.0]) if abs(ez[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        v = tmp - np.dot(tmp, ez) * ez
    ex = v / np.linalg.norm(v)
    return np.stack([ex, np.cross(ez, ex), ez])


def _ref_pair_frames(mol):
    X = mol.coords
    el = np.array([guess.ELEM[s] for s in mol.symbols])
    n = len(el)
    D = np.linalg.norm(X[:, None] - X[None], axis=-1)
    pairs, frames, feats = [], [], []
    for a in range(n):
        for b in range(n):
            if (a != b and (el[a], a) > (el[b], b)) or D[a, b] > guess.PAIR_CUTOFF:
                continue
            mid = 0.5 * (X[a] + X[b])
            others = [c for c in range(n) if c != a and c != b]
            dm = np.linalg.norm(X[others] - mid, axis=1) if others else np.zeros(0)
            order = [others[i] for i in np.argsort(dm, kind="stable")]
            if a != b:
                ez, ref = X[b] - X[a], (X[order[0]] - mid if order else np.array([0.0, 0.0, 1.0]))
            else:
                ez = X[order[0]] - X[a] if order else np.array([0.0, 0.0, 1.0])
                ref = X[order[1]] - X[a] if len(order) > 1 else np.array([1.0, 0.0, 0.0])
            R = _ref_frame(ez, ref)
            f = np.zeros(guess.NFEAT, dtype=np.float32)
            f[el[a]] = f[3 + el[b]] = 1.0
            f[6] = 1.0 if a == b else 0.0
            f[7] = D[a, b] / 5.0
            f[8:8 + len(guess.RBF)] = np.exp(-((D[a, b] - guess.RBF) ** 2))
            o = 8 + len(guess.RBF)
            for k, c in enumerate(order[:guess.NNB]):
                loc = R @ (X[c] - mid)
                f[o + 7 * k:o + 7 * k + 3] = loc / 5.0
                f[o + 7 * k + 3] = 1.0 / (1.0 + np.linalg.norm(loc))
                f[o + 7 * k + 4 + el[c]] = 1.0
            pairs.append((a, b))
            frames.append(R)
            feats.append(f)
    return pairs, frames, np.array(feats, dtype=np.float32).reshape(-1, guess.NFEAT)


def _ref_blocks(D, bas, pairs, frames, Y, nbf):
    sh = guess.atom_shells(bas)
    T = np.zeros((len(pairs), guess.NOUT))
    Dout = np.zeros((nbf, nbf))
    for k, ((a, b), R) in enumerate(zip(pairs, frames)):
        Ma, Mb = guess.atom_M(sh[a]["ls"], R), guess.atom_M(sh[b]["ls"], R)
        na, nb = Ma.shape[0], Mb.shape[0]
        fa, fb = sh[a]["first"], sh[b]["first"]
        t = np.zeros((guess.MAXB, guess.MAXB))
        t[:na, :nb] = Ma.T @ D[fa:fa + na, fb:fb + nb] @ Mb
        T[k] = t.ravel()
        loc = Y[k].reshape(guess.MAXB, guess.MAXB)[:na, :nb].astype(np.float64)
        if a == b:
            loc = 0.5 * (loc + loc.T)
        blk = np.linalg.solve(Ma.T, np.linalg.solve(Mb.T, loc.T).T)
        Dout[fa:fa + na, fb:fb + nb] = blk
        if a != b:
            Dout[fb:fb + nb, fa:fa + na] = blk.T
    return T, Dout


def test_vectorised_preparation_matches_pairwise_definition():
    table = molgen.basis_set("dz", 0)
    r = np.random.Generator(np.random.PCG64(11))
    mols = molgen.scf_conformations(6, 3) + [molgen.water_chain_cluster(1, r), molgen.water_chain_cluster(2, r),
                                             molgen.water_sphere_cluster(24, r)]
    for mol in mols:
        bas = molgen.make_basis(mol, table)
        n = molgen.nbf(bas)
        p0, f0, x0 = _ref_pair_frames(mol)
        p1, f1, x1 = guess.pair_frames(mol)
        assert p0 == p1
        assert np.abs(np.array(f0) - np.array(f1)).max() < 1e-13
        assert np.abs(x0 - x1).max() < 1e-6
        D = r.uniform(-1, 1, (n, n))
        D = D + D.T
        Y = r.normal(size=(len(p0), guess.NOUT)).astype(np.float32)
        T0, D0 = _ref_blocks(D, bas, p0, f0, Y, n)
        T1, _ = guess.blocks_to_local(D, mol, bas, p1, f1)
        D1 = guess.local_to_density(Y, mol, bas, p1, f1, n)
        assert np.abs(T0.astype(np.float32) - T1).max() <= 1e-5 * max(1.0, np.abs(T0).max())
        assert np.abs(D0 - D1).max() <= 1e-11 * max(1.0, np.abs(D0).max())
