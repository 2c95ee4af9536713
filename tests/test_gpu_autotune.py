"""Measured per-class-pair schedules (fock_autotune): every forced schedule
and every isolated plan gives the oracle's J and K within 1e-10; the tuned
options are valid, and the builds they plan (single and batched) keep
parity."""
import numpy as np
import pytest

import molgen
import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    import paper_2407_21445_gb300 as fk
    return torch, fk


def _rand_basis(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    bas = molgen.random_shells(rng, [0, 1, 2, 3, 0, 1, 2, 0, 1], spread=3.5, kmax=3)
    n = oracle.nbf(bas)
    D = rng.uniform(-1, 1, (n, n))
    return bas, 0.5 * (D + D.T)


def _jk(env, basis, D, tau, opts):
    torch, fk = env
    b = fk.JKBuilder(basis, tau, opts)
    J, K = b.build(torch.tensor(D, device="cuda", dtype=torch.float64))
    torch.cuda.synchronize()
    assert fk.fock_stream_status() == 0
    out = J.cpu().numpy(), K.cpu().numpy(), fk.fock_kernels_per_build(b.handle)
    b.close()
    return out


@pytest.mark.parametrize("cand", [-1, 1, 2, 4, 8, 16, 32])
def test_forced_schedule_isolated(env, cand):
    """Every class pair forced to one candidate, each class pair in launches
    of its own."""
    torch, fk = env
    bas, D = _rand_basis(410)
    Jo, Ko = oracle.jk(bas, D, 1e-11)
    sched = {(a, b): cand for a in range(fk.NCLASS) for b in range(a, fk.NCLASS)}
    o = fk.make_opts(schedule=sched)
    o.tune_isolate = 1
    J, K, nk = _jk(env, bas, D, 1e-11, o)
    assert np.abs(J - Jo).max() <= TOL and np.abs(K - Ko).max() <= TOL
    o.tune_isolate = 0
    J2, K2, nk2 = _jk(env, bas, D, 1e-11, o)
    assert np.abs(J2 - Jo).max() <= TOL and np.abs(K2 - Ko).max() <= TOL
    assert nk >= nk2


def test_autotune_single(env):
    torch, fk = env
    p = molgen.problem(0)
    Dt = torch.tensor(p.D, device="cuda", dtype=torch.float64)
    o, ms, pair = fk.fock_autotune([p.basis], [Dt], p.tau, None, reps=2)
    assert ms[0] > 0 and ms[1] > 0 and o.tune_isolate == 0
    assert pair and all(a <= b for a, b in pair) and sum(pair.values()) < 3 * ms[0]
    assert set(fk.schedule_of(o).values()) <= {-1, 1, 2, 4, 8, 16, 32}
    J, K, _ = _jk(env, p.basis, p.D, p.tau, o)
    Jo, Ko = oracle.jk(p.basis, p.D, p.tau)
    assert np.abs(J - Jo).max() <= TOL and np.abs(K - Ko).max() <= TOL


def test_autotune_batched_and_cache(env, tmp_path):
    torch, fk = env
    from paper_2407_21445_gb300 import autotune
    probs = molgen.batch_problems(3, seed=7, kind="dz")
    bases = [q.basis for q in probs]
    Ds = [torch.tensor(q.D, device="cuda", dtype=torch.float64) for q in probs]
    tau = probs[0].tau
    cache = str(tmp_path / "tune.json")
    o, rec = autotune.tuned_opts(bases, Ds, tau, cache=cache, reps=1)
    assert not rec["cached"] and rec["ms_base"] > 0
    o2, rec2 = autotune.tuned_opts(bases, Ds, tau, cache=cache)
    assert rec2["cached"] and fk.schedule_of(o2) == fk.schedule_of(o)
    hs = [fk.fock_shellpairs_build(b, tau, o) for b in bases]
    Js = [torch.empty_like(d) for d in Ds]
    Ks = [torch.empty_like(d) for d in Ds]
    fk.fock_build_jk_batched(hs, Ds, tau, Js, Ks)
    torch.cuda.synchronize()
    assert fk.fock_stream_status() == 0
    small = sorted(range(3), key=lambda i: oracle.nbf(probs[i].basis))[:2]
    for i in small:
        q, J, K = probs[i], Js[i], Ks[i]
        Jo, Ko = oracle.jk(q.basis, q.D, tau)
        assert np.abs(J.cpu().numpy() - Jo).max() <= TOL and np.abs(K.cpu().numpy() - Ko).max() <= TOL
    for h in hs:
        fk.fock_shellpairs_free(h)
