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
