"""Batched build: many molecules of uneven size in one pass (one launch per
class tier over all molecules, captured in a CUDA graph) must reproduce the
per-molecule build and the oracle, on first and replayed calls."""
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


def _run(env, probs, opts=None, scale=1.0):
    torch, fk = env
    builders = [fk.JKBuilder(p.basis, p.tau, opts) for p in probs]
    Ds = [torch.tensor(scale * p.D, device="cuda") for p in probs]
    Js = [torch.empty_like(d) for d in Ds]
    Ks = [torch.empty_like(d) for d in Ds]
    fk.fock_build_jk_batched([b.handle for b in builders], Ds, probs[0].tau, Js, Ks)
    torch.cuda.synchronize()
    assert fk.fock_stream_status() == 0
    return builders, Ds, Js, Ks


def test_batched_matches_single_and_replay(env):
    torch, fk = env
    probs = molgen.batch_problems(12, seed=1)
    builders, Ds, Js, Ks = _run(env, probs)
    for b, D, J, K in zip(builders, Ds, Js, Ks):
        J1, K1 = b.build(D)
        torch.cuda.synchronize()
        assert float((J - J1).abs().max()) < 1e-12 and float((K - K1).abs().max()) < 1e-12
    # replay of the captured graph with new densities
    Ds2 = [0.5 * d for d in Ds]
    Js2 = [torch.empty_like(d) for d in Ds]
    Ks2 = [torch.empty_like(d) for d in Ds]
    fk.fock_build_jk_batched([b.handle for b in builders], Ds2, probs[0].tau, Js2, Ks2)
    torch.cuda.synchronize()
    for b, D, J, K in zip(builders, Ds2, Js2, Ks2):
        J1, K1 = b.build(D)
        torch.cuda.synchronize()
        assert float((J - J1).abs().max()) < 1e-12 and float((K - K1).abs().max()) < 1e-12


def test_batched_against_oracle(env):
    probs = molgen.batch_problems(6, seed=2)
    small = sorted(probs, key=lambda p: p.nbf)[:3]
    builders, Ds, Js, Ks = _run(env, small)
    for p, J, K in zip(small, Js, Ks):
        Jo, Ko = oracle.jk(p.basis, p.D, p.tau)
        assert np.abs(J.cpu().numpy() - Jo).max() <= 1e-10
        assert np.abs(K.cpu().numpy() - Ko).max() <= 1e-10


def test_batched_mixed_against_oracle(env):
    torch, fk = env
    probs = sorted(molgen.batch_problems(6, seed=3), key=lambda p: p.nbf)[:3]
    builders, Ds, Js, Ks = _run(env, probs, fk.make_opts(precision=fk.FOCK_MIXED, fp32_cutoff=1e-5))
    for p, J, K in zip(probs, Js, Ks):
        Jo, Ko = oracle.jk(p.basis, p.D, p.tau)
        assert np.abs(J.cpu().numpy() - Jo).max() <= 1e-7
        assert np.abs(K.cpu().numpy() - Ko).max() <= 1e-7


def test_batched_rejects_mismatched_options(env):
    torch, fk = env
    probs = molgen.batch_problems(2, seed=4)
    b1 = fk.JKBuilder(probs[0].basis, probs[0].tau)
    b2 = fk.JKBuilder(probs[1].basis, probs[1].tau, fk.make_opts(precision=fk.FOCK_MIXED))
    Ds = [torch.tensor(p.D, device="cuda") for p in probs]
    with pytest.raises(fk.FockError):
        fk.fock_build_jk_batched([b1.handle, b2.handle], Ds, probs[0].tau, [torch.empty_like(d) for d in Ds],
                                 [torch.empty_like(d) for d in Ds])
