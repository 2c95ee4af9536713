"""Mixed-precision path: quartets whose density-weighted Schwarz bound is
below the FP32 cutoff are evaluated in FP32 (J/K accumulated in FP64);
J and K must match the FP64 oracle within max-abs 1e-7 and the scalar
tr(D(2J-K)) within 1e-6 Eh."""
import numpy as np
import pytest

import molgen
import oracle

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-7
TOL_TR = 1e-6


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    import paper_2407_21445_gb300 as fk
    return torch, fk


def mixed_jk(env, basis, D, tau, cutoff=1e-5, **kw):
    torch, fk = env
    b = fk.JKBuilder(basis, tau, fk.make_opts(precision=fk.FOCK_MIXED, fp32_cutoff=cutoff, **kw))
    Dt = torch.tensor(D, device="cuda", dtype=torch.float64)
    J, K = b.build(Dt)
    torch.cuda.synchronize()
    assert fk.fock_stream_status() == 0
    st = b.stats(D)
    return J.cpu().numpy(), K.cpu().numpy(), st


def check(J, K, Jo, Ko, D):
    ej, ek = np.abs(J - Jo).max(), np.abs(K - Ko).max()
    tr = abs(np.sum(D * (2 * J - K)) - np.sum(D * (2 * Jo - Ko)))
    assert ej <= TOL_MIXED and ek <= TOL_MIXED and tr <= TOL_TR, (ej, ek, tr)
    return ej, ek, tr


def test_mixed_water_trimer(env):
    p = molgen.problem(0)
    J, K, st = mixed_jk(env, p.basis, p.D, p.tau)
    Jo, Ko = oracle.jk(p.basis, p.D, p.tau)
    check(J, K, Jo, Ko, p.D)
    assert st["quartets_fp32"] > 0


def test_mixed_alkane_full(env):
    p = molgen.problem(1)
    J, K, st = mixed_jk(env, p.basis, p.D, p.tau)
    Jo, Ko = oracle.jk(p.basis, p.D, p.tau)
    ej, ek, tr = check(J, K, Jo, Ko, p.D)
    assert st["quartets_fp32"] > 0.3 * st["quartets_evaluated"]
    print(f"C20H42 mixed: max|dJ|={ej:.2e} max|dK|={ek:.2e} |dtr|={tr:.2e} fp32 share "
          f"{st['quartets_fp32'] / st['quartets_evaluated']:.2f}")


def test_mixed_cutoff_zero_is_fp64(env):
    """A zero cutoff sends every quartet down the FP64 path (1e-10 parity)."""
    p = molgen.problem(0)
    J, K, st = mixed_jk(env, p.basis, p.D, p.tau, cutoff=0.0)
    Jo, Ko = oracle.jk(p.basis, p.D, p.tau)
    assert st["quartets_fp32"] == 0
    assert np.abs(J - Jo).max() <= 1e-10 and np.abs(K - Ko).max() <= 1e-10


def test_mixed_random_f_basis(env):
    rng = np.random.Generator(np.random.PCG64(300))
    bas = molgen.random_shells(rng, [0, 1, 2, 3, 0, 1, 2, 1, 0, 0], spread=4.0, kmax=4)
    n = oracle.nbf(bas)
    D = rng.uniform(-1, 1, (n, n))
    D = 0.5 * (D + D.T)
    J, K, st = mixed_jk(env, bas, D, 1e-11)
    Jo, Ko = oracle.jk(bas, D, 1e-11)
    check(J, K, Jo, Ko, D)


def test_mixed_water64_blocks(env):
    p = molgen.problem(2)
    J, K, st = mixed_jk(env, p.basis, p.D, p.tau)
    ls = p.basis["l"]
    offs = np.concatenate([[0], np.cumsum([oracle.ncart(int(l)) for l in ls])])
    ns = len(ls)
    rng = np.random.Generator(np.random.PCG64(9))
    pairs = [(0, 0), (ns - 1, 0)] + [tuple(int(x) for x in rng.integers(0, ns, 2)) for _ in range(4)]
    Jb, Kb = oracle.jk_blocks(p.basis, p.D, pairs, p.tau)
    for (a, b), jb, kb in zip(pairs, Jb, Kb):
        assert np.abs(J[offs[a]:offs[a + 1], offs[b]:offs[b + 1]] - jb).max() <= TOL_MIXED
        assert np.abs(K[offs[a]:offs[a + 1], offs[b]:offs[b + 1]] - kb).max() <= TOL_MIXED


@pytest.mark.parametrize("group", [0, 1, 4, 32])
def test_mixed_group_kernels(env, group):
    """Every class pair on the group-cooperative kernels (no register
    kernels), for several group sizes: their FP64 and FP32 parts."""
    rng = np.random.Generator(np.random.PCG64(301 + group))
    bas = molgen.random_shells(rng, [0, 1, 2, 3, 0, 1, 2, 0], spread=6.0, kmax=3)
    n = oracle.nbf(bas)
    D = rng.uniform(-1, 1, (n, n))
    D = 0.5 * (D + D.T)
    J, K, st = mixed_jk(env, bas, D, 1e-11, cutoff=1e-4, reg_max_L=-1, group_override=group)
    Jo, Ko = oracle.jk(bas, D, 1e-11)
    check(J, K, Jo, Ko, D)
    assert st["quartets_fp32"] > 0


def test_mixed_kernel_count(env):
    """A mixed build launches one extra kernel per group-kernel tier (its
    FP32 part); with every class pair on register kernels the counts agree."""
    torch, fk = env
    p = molgen.problem(0)
    n64 = fk.JKBuilder(p.basis, p.tau, fk.make_opts(precision=fk.FOCK_FP64))
    nmx = fk.JKBuilder(p.basis, p.tau, fk.make_opts(precision=fk.FOCK_MIXED))
    k64, kmx = fk.fock_kernels_per_build(n64.handle), fk.fock_kernels_per_build(nmx.handle)
    assert kmx > k64  # the trimer has d shells, so group tiers exist
    b = molgen.single_shell_basis([(1, np.zeros(3), np.array([1.0]), np.array([1.0])),
                                   (0, np.array([0.0, 0.0, 1.5]), np.array([0.8]), np.array([1.0]))])
    r64 = fk.JKBuilder(b, 1e-12, fk.make_opts(precision=fk.FOCK_FP64))
    rmx = fk.JKBuilder(b, 1e-12, fk.make_opts(precision=fk.FOCK_MIXED))
    assert fk.fock_kernels_per_build(r64.handle) == fk.fock_kernels_per_build(rmx.handle)
    for x in (n64, nmx, r64, rmx):
        x.close()


@pytest.mark.parametrize("group", [0, 1, 8, 32])
def test_mixed_primitive_tails(env, group):
    """Inside a quartet whose bound is at or above the cutoff, every primitive
    quartet whose own bound G_[ab] G_[cd] Dmax is below it runs in FP32 (in the
    register kernels, group = 0, and in the group kernels forced to 1, 8 and 32
    lanes per quartet).  A cutoff of 1e-3 sends most primitive quartets of the
    FP64 quartets of this contracted d/f basis down that path."""
    rng = np.random.Generator(np.random.PCG64(301))
    bas = molgen.random_shells(rng, [0, 0, 1, 2, 3, 1, 0, 2], spread=3.0, kmax=6)
    n = oracle.nbf(bas)
    D = rng.uniform(-1, 1, (n, n))
    D = 0.5 * (D + D.T)
    J, K, st = mixed_jk(env, bas, D, 1e-11, cutoff=1e-3, group_override=group)
    Jo, Ko = oracle.jk(bas, D, 1e-11)
    ej, ek, tr = check(J, K, Jo, Ko, D)
    share_q = st["quartets_fp32"] / st["quartets_evaluated"]
    share_f = st["flops_model_fp32"] / st["flops_model"]
    print(f"group {group}: max|dJ|={ej:.2e} max|dK|={ek:.2e} FP32 quartets {share_q:.2f}, FP32 flops {share_f:.2f}")


def test_mixed_tails_alkane_stats(env):
    """C20H42 with the default cutoff: the primitive tails move FP32 work into
    the FP64 quartets (modelled FP32 flop share above the quartet share)."""
    p = molgen.problem(1)
    J, K, st = mixed_jk(env, p.basis, p.D, p.tau)
    Jo, Ko = oracle.jk(p.basis, p.D, p.tau)
    check(J, K, Jo, Ko, p.D)
    assert st["flops_model_fp32"] / st["flops_model"] > st["quartets_fp32"] / st["quartets_evaluated"]
