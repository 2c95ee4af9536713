"""FP64 one-electron integrals on the GPU (fock_one_electron, MMD) against the
oracle's Obara-Saika S, T, V."""
import numpy as np
import pytest

import molgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    import paper_2407_21445_gb300 as fk
    return torch, fk


@pytest.mark.parametrize("case", ["trimer", "random_f"])
def test_one_electron_matches_oracle(env, case):
    torch, fk = env
    if case == "trimer":
        p = molgen.problem(0)
        bas, Z, xyz = p.basis, p.mol.Z.astype(float), p.mol.coords
    else:
        rng = np.random.Generator(np.random.PCG64(41))
        bas = molgen.random_shells(rng, [0, 1, 2, 3, 2, 1, 0], spread=2.0, kmax=4)
        Z, xyz = np.array([1.0, 8.0, 6.0]), rng.uniform(-2, 2, (3, 3))
    S, T, V = fk.fock_one_electron(bas, Z, xyz)
    So, To, Vo = oracle.overlap(bas), oracle.kinetic(bas), oracle.nuclear(bas, Z, xyz)
    assert np.abs(S.cpu().numpy() - So).max() < 1e-12
    assert np.abs(T.cpu().numpy() - To).max() < 1e-11
    assert np.abs(V.cpu().numpy() - Vo).max() < 1e-11
