"""GPU parity: libfock.so (called through the C ABI via the ctypes binding)
against the CPU oracle on the same seeded inputs.

Tolerances: FP64 path max-abs element error 1e-10 on J and K, and
|tr(D(2J - K))| within 1e-6 Eh.  Screening (Schwarz + six-block density
test, Sec. 3.2) and primitive-pair pruning use the same rules on both sides.
"""
import numpy as np
import pytest

import molgen
import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-10
TOL_TR = 1e-6


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return t


@pytest.fixture(scope="module")
def fk():
    import paper_2407_21445_gb300 as m
    return m


def gpu_jk(fk, torch, basis, D, tau, group=0, prune=1e-3):
    b = fk.JKBuilder(basis, tau, fk.make_opts(group_override=group, prune_eps=prune))
    Dt = torch.tensor(D, device="cuda", dtype=torch.float64)
    J, K = b.build(Dt)
    torch.cuda.synchronize()
    st = fk.fock_stream_status()
    assert st == 0, fk.fock_status_string(st)
    return J.cpu().numpy(), K.cpu().numpy(), b


def compare(J, K, Jo, Ko, D):
    ej, ek = np.abs(J - Jo).max(), np.abs(K - Ko).max()
    tr = abs(np.sum(D * (2 * J - K)) - np.sum(D * (2 * Jo - Ko)))
    assert ej <= TOL and ek <= TOL and tr <= TOL_TR, (ej, ek, tr)
    assert np.abs(J - J.T).max() == 0.0 and np.abs(K - K.T).max() == 0.0
    return ej, ek, tr


@pytest.fixture(scope="module")
def c0():
    p = molgen.problem(0)
    Jo, Ko = oracle.jk(p.basis, p.D, p.tau)
    return p, Jo, Ko


def test_water_trimer_full(fk, torch, c0):
    p, Jo, Ko = c0
    J, K, _ = gpu_jk(fk, torch, p.basis, p.D, p.tau)
    compare(J, K, Jo, Ko, p.D)


@pytest.mark.parametrize("group", [1, 2, 4, 8, 16, 32])
def test_water_trimer_every_group_size(fk, torch, c0, group):
    p, Jo, Ko = c0
    J, K, _ = gpu_jk(fk, torch, p.basis, p.D, p.tau, group=group)
    compare(J, K, Jo, Ko, p.D)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_shells_all_classes_to_f(fk, torch, seed):
    """Random centres and contractions, l = 0..3: every class pair up to (ff|ff)."""
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    ls = [0, 1, 2, 3, 0, 1, 2, 3, 1, 0, 2]
    bas = molgen.random_shells(rng, ls, spread=2.5, kmax=4)
    n = oracle.nbf(bas)
    D = rng.uniform(-1, 1, (n, n))
    D = 0.5 * (D + D.T)
    tau = 1e-11
    Jo, Ko = oracle.jk(bas, D, tau)
    J, K, _ = gpu_jk(fk, torch, bas, D, tau)
    compare(J, K, Jo, Ko, D)


def test_no_pruning_matches(fk, torch):
    rng = np.random.Generator(np.random.PCG64(7))
    bas = molgen.random_shells(rng, [0, 1, 2, 0, 1, 3], spread=2.0, kmax=3)
    n = oracle.nbf(bas)
    D = rng.uniform(-1, 1, (n, n))
    D = D + D.T
    Jo, Ko = oracle.jk(bas, D, 1e-12, eps_prune=0.0)
    J, K, _ = gpu_jk(fk, torch, bas, D, 1e-12, prune=0.0)
    compare(J, K, Jo, Ko, D)


@pytest.fixture(scope="module")
def c1_gpu(fk, torch):
    p = molgen.problem(1)
    J, K, b = gpu_jk(fk, torch, p.basis, p.D, p.tau)
    return p, J, K, b


def test_alkane_c20h42_full(fk, torch, c1_gpu):
    """The benchmark workload, element by element against the full oracle."""
    p, J, K, _ = c1_gpu
    Jo, Ko = oracle.jk(p.basis, p.D, p.tau)
    compare(J, K, Jo, Ko, p.D)


def test_alkane_work_counts_match_oracle(fk, torch, c1_gpu):
    p, _, _, b = c1_gpu
    st = b.stats(p.D)
    cnt = oracle.count(p.basis, p.D, p.tau)
    assert st["quartets_schwarz"] == cnt["quartets_schwarz"]
    assert st["eris_schwarz"] == cnt["eris_schwarz"]
    assert st["quartets_evaluated"] == cnt["quartets_density"]
    assert st["eris_evaluated"] == cnt["eris_density"]


def test_water64_sampled_blocks(fk, torch):
    """(H2O)64 sphere (1216 functions): seeded shell-pair blocks of J and K
    computed one by one by the oracle."""
    p = molgen.problem(2)
    J, K, _ = gpu_jk(fk, torch, p.basis, p.D, p.tau)
    ls = p.basis["l"]
    offs = np.concatenate([[0], np.cumsum([oracle.ncart(int(l)) for l in ls])])
    rng = np.random.Generator(np.random.PCG64(3))
    ns = len(ls)
    pairs = [(0, 0), (5, 5), (ns - 1, 0)]
    pairs += [tuple(int(x) for x in rng.integers(0, ns, 2)) for _ in range(5)]
    d_shells = [s for s in range(ns) if ls[s] == 2]
    pairs += [(d_shells[0], d_shells[-1]), (d_shells[3], 2)]
    Jb, Kb = oracle.jk_blocks(p.basis, p.D, pairs, p.tau)
    for (a, b), jb, kb in zip(pairs, Jb, Kb):
        ej = np.abs(J[offs[a]:offs[a + 1], offs[b]:offs[b + 1]] - jb).max()
        ek = np.abs(K[offs[a]:offs[a + 1], offs[b]:offs[b + 1]] - kb).max()
        assert ej <= TOL and ek <= TOL, (a, b, ej, ek)


def test_repeat_is_reproducible(fk, torch, c0):
    p, _, _ = c0
    J1, K1, b = gpu_jk(fk, torch, p.basis, p.D, p.tau)
    Dt = torch.tensor(p.D, device="cuda")
    J2, K2 = b.build(Dt)
    assert np.abs(J2.cpu().numpy() - J1).max() < 1e-13 and np.abs(K2.cpu().numpy() - K1).max() < 1e-13


def test_everything_screened_gives_zero(fk, torch, c0):
    p, _, _ = c0
    b = fk.JKBuilder(p.basis, p.tau)
    Dt = torch.tensor(p.D, device="cuda")
    J, K = b.build(Dt, tau=1e6)
    torch.cuda.synchronize()
    assert float(J.abs().max()) == 0.0 and float(K.abs().max()) == 0.0


def test_single_s_shell(fk, torch):
    """One normalised s Gaussian: J = K = 2 sqrt(a/pi) D_00."""
    bas = molgen.single_shell_basis([(0, [0.3, 0.1, -0.2], [1.7], [1.0])])
    J, K, _ = gpu_jk(fk, torch, bas, np.array([[0.7]]), 1e-12)
    ref = 2 * np.sqrt(1.7 / np.pi) * 0.7
    assert abs(J[0, 0] - ref) < 1e-14 and abs(K[0, 0] - ref) < 1e-14


def test_threshold_below_build_is_rejected(fk, torch, c0):
    p, _, _ = c0
    b = fk.JKBuilder(p.basis, p.tau)
    Dt = torch.tensor(p.D, device="cuda")
    with pytest.raises(fk.FockError) as e:
        b.build(Dt, tau=p.tau / 10)
    assert e.value.status == 1


def test_nonfinite_density_sets_status(fk, torch, c0):
    p, _, _ = c0
    b = fk.JKBuilder(p.basis, p.tau)
    D = p.D.copy()
    D[3, 4] = D[4, 3] = np.nan
    Dt = torch.tensor(D, device="cuda")
    b.build(Dt)
    assert fk.fock_stream_status() == 3
    assert fk.fock_stream_status() == 0  # cleared after reading
