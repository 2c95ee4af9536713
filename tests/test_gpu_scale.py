"""One mixed-precision J/K build of the 1,002-atom water cluster (H2O)334
(6,346 basis functions) for scale, checked on sampled shell-pair blocks
against the FP64 oracle (max-abs 1e-7).  Minutes of GPU and oracle time, so
it runs only when FOCK_SCALE=1:

    FOCK_SCALE=1 python -m pytest tests/test_gpu_scale.py -m gpu -s

The second test runs the batched workload at its full size (256 TZ molecules).
"""
import os
import time

import numpy as np
import pytest

import molgen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow,
              pytest.mark.skipif(os.environ.get("FOCK_SCALE") != "1", reason="set FOCK_SCALE=1 (minutes)")]

TOL_MIXED = 1e-7


def test_water334_mixed_build_blocks():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    import paper_2407_21445_gb300 as fk
    p = molgen.problem(2, waters=334)
    t0 = time.perf_counter()
    b = fk.JKBuilder(p.basis, p.tau, fk.make_opts(precision=fk.FOCK_MIXED, fp32_cutoff=1e-5))
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    D = torch.tensor(p.D, device="cuda", dtype=torch.float64)
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    b.build(D, J, K)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e)
    assert fk.fock_stream_status() == 0
    Jh, Kh = J.cpu().numpy(), K.cpu().numpy()
    ls = p.basis["l"]
    offs = np.concatenate([[0], np.cumsum([oracle.ncart(int(l)) for l in ls])])
    ns = len(ls)
    rng = np.random.Generator(np.random.PCG64(334))
    pairs = [(0, 0), (ns - 1, ns // 2)] + [tuple(int(x) for x in rng.integers(0, ns, 2)) for _ in range(2)]
    Jb, Kb = oracle.jk_blocks(p.basis, p.D, pairs, p.tau)
    errs = []
    for (a, bb), jb, kb in zip(pairs, Jb, Kb):
        ej = np.abs(Jh[offs[a]:offs[a + 1], offs[bb]:offs[bb + 1]] - jb).max()
        ek = np.abs(Kh[offs[a]:offs[a + 1], offs[bb]:offs[bb + 1]] - kb).max()
        errs.append(max(ej, ek))
    assert np.isfinite(Jh).all() and np.isfinite(Kh).all()
    assert np.abs(Jh - Jh.T).max() == 0.0 and np.abs(Kh - Kh.T).max() == 0.0
    print(f"(H2O)334 nbf={p.nbf} plan {t_plan:.1f} s, mixed J+K build {ms / 1e3:.2f} s, "
          f"kernels {fk.fock_kernels_per_build(b.handle)}, sampled-block max-abs error vs oracle {max(errs):.2e}")
    assert max(errs) <= TOL_MIXED


def test_batched_256_tz_one_build():
    """The batched workload at its full size: 256 molecules of 5-40 atoms,
    triple-zeta-shaped basis up to f, one fock_build_jk_batched call (FP64),
    checked against the oracle on the two smallest molecules (every element)
    and on sampled blocks of the largest."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    import paper_2407_21445_gb300 as fk
    probs = molgen.batch_problems(256)
    tau = probs[0].tau
    t0 = time.perf_counter()
    hs = [fk.fock_shellpairs_build(p.basis, tau) for p in probs]
    t_plan = time.perf_counter() - t0
    Ds = [torch.tensor(p.D, device="cuda", dtype=torch.float64) for p in probs]
    Js = [torch.empty_like(d) for d in Ds]
    Ks = [torch.empty_like(d) for d in Ds]
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    fk.fock_build_jk_batched(hs, Ds, tau, Js, Ks)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e)
    assert fk.fock_stream_status() == 0
    nbf = [p.nbf for p in probs]
    order = sorted(range(len(probs)), key=lambda i: nbf[i])
    for i in order[:2]:
        Jo, Ko = oracle.jk(probs[i].basis, probs[i].D, tau)
        assert np.abs(Js[i].cpu().numpy() - Jo).max() <= 1e-10 and np.abs(Ks[i].cpu().numpy() - Ko).max() <= 1e-10
    big = order[-1]
    p = probs[big]
    ls = p.basis["l"]
    offs = np.concatenate([[0], np.cumsum([oracle.ncart(int(l)) for l in ls])])
    rng = np.random.Generator(np.random.PCG64(256))
    pairs = [tuple(int(x) for x in rng.integers(0, len(ls), 2)) for _ in range(3)]
    Jb, Kb = oracle.jk_blocks(p.basis, p.D, pairs, tau)
    J, K = Js[big].cpu().numpy(), Ks[big].cpu().numpy()
    for (a, b), jb, kb in zip(pairs, Jb, Kb):
        assert np.abs(J[offs[a]:offs[a + 1], offs[b]:offs[b + 1]] - jb).max() <= 1e-10
        assert np.abs(K[offs[a]:offs[a + 1], offs[b]:offs[b + 1]] - kb).max() <= 1e-10
    print(f"256 TZ molecules, {sum(nbf)} functions: plans {t_plan:.1f} s, one batched FP64 build {ms / 1e3:.2f} s")
    for h in hs:
        fk.fock_shellpairs_free(h)
