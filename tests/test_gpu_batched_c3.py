"""A 32-molecule batch of the batched workload (molecules of 5-40 atoms,
triple-zeta-shaped basis up to f) through fock_build_jk_batched, in FP64 and
in mixed precision: the three smallest molecules against the oracle element
by element, sampled shell-pair blocks of the largest one by one (FP64 1e-10,
mixed 1e-7 and |d tr(D(2J-K))| <= 1e-6 on the full molecules)."""
import numpy as np
import pytest

import molgen
import oracle

pytestmark = pytest.mark.gpu

NMOL = 32


@pytest.fixture(scope="module")
def batch():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    import paper_2407_21445_gb300 as fk
    probs = molgen.batch_problems(NMOL)
    nbf = [p.nbf for p in probs]
    order = sorted(range(NMOL), key=lambda i: nbf[i])
    small = order[:3]
    big = order[-1]
    p = probs[big]
    ls = p.basis["l"]
    rng = np.random.Generator(np.random.PCG64(32))
    pairs = [(0, 0)] + [tuple(int(x) for x in rng.integers(0, len(ls), 2)) for _ in range(3)]
    ref_small = {i: oracle.jk(probs[i].basis, probs[i].D, probs[i].tau) for i in small}
    ref_big = oracle.jk_blocks(p.basis, p.D, pairs, p.tau)
    return torch, fk, probs, small, big, pairs, ref_small, ref_big


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-7)])
def test_batched_32_tz_molecules(batch, precision, tol):
    torch, fk, probs, small, big, pairs, ref_small, ref_big = batch
    tau = probs[0].tau
    opts = fk.make_opts(precision=precision)
    hs = [fk.fock_shellpairs_build(p.basis, tau, opts) for p in probs]
    Ds = [torch.tensor(p.D, device="cuda", dtype=torch.float64) for p in probs]
    Js = [torch.empty_like(d) for d in Ds]
    Ks = [torch.empty_like(d) for d in Ds]
    fk.fock_build_jk_batched(hs, Ds, tau, Js, Ks)
    torch.cuda.synchronize()
    assert fk.fock_stream_status() == 0
    worst = 0.0
    for i in small:
        Jo, Ko = ref_small[i]
        J, K = Js[i].cpu().numpy(), Ks[i].cpu().numpy()
        e = max(np.abs(J - Jo).max(), np.abs(K - Ko).max())
        tr = abs(np.sum(probs[i].D * (2 * J - K)) - np.sum(probs[i].D * (2 * Jo - Ko)))
        assert e <= tol and tr <= 1e-6, (i, e, tr)
        worst = max(worst, e)
    p = probs[big]
    offs = np.concatenate([[0], np.cumsum([oracle.ncart(int(l)) for l in p.basis["l"]])])
    J, K = Js[big].cpu().numpy(), Ks[big].cpu().numpy()
    for (a, b), jb, kb in zip(pairs, *ref_big):
        e = max(np.abs(J[offs[a]:offs[a + 1], offs[b]:offs[b + 1]] - jb).max(),
                np.abs(K[offs[a]:offs[a + 1], offs[b]:offs[b + 1]] - kb).max())
        assert e <= tol, ((a, b), e)
        worst = max(worst, e)
    print(f"{NMOL} TZ molecules, precision {precision}: worst max-abs error vs oracle {worst:.2e}")
    for h in hs:
        fk.fock_shellpairs_free(h)
