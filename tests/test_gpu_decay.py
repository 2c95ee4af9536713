"""J-only and K-only builds (J or K passed as NULL) and the heuristic
decay-bound exchange mode (Sec. 4.3.1), through the C ABI on the GPU.

J-only / K-only builds weigh a quartet by the density blocks that feed the
part they build, exactly as the oracle's modes 3 and 4 do: FP64 parity
1e-10.  The decay-bound mode is a heuristic (the paper bounds its effect only
empirically): its error against the exact mode is measured and held to a
stated bound.  Its fit (H, Lambda) and radii must equal the oracle's."""
import numpy as np
import pytest

import molgen
import oracle
from oracle import decay

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    import paper_2407_21445_gb300 as fk
    return torch, fk


def _dev(torch, D):
    return torch.tensor(D, device="cuda", dtype=torch.float64)


@pytest.mark.parametrize("case", ["trimer", "c10", "random_f"])
def test_j_only_and_k_only_match_oracle_modes(env, case):
    torch, fk = env
    if case == "trimer":
        p = molgen.problem(0)
        bas, D, tau = p.basis, p.D, p.tau
    elif case == "c10":
        p = molgen.problem(1, carbons=10)
        bas, D, tau = p.basis, p.D, p.tau
    else:
        rng = np.random.Generator(np.random.PCG64(310))
        bas = molgen.random_shells(rng, [0, 1, 2, 3, 0, 1, 2, 0], spread=3.5, kmax=4)
        n = oracle.nbf(bas)
        D = rng.uniform(-1, 1, (n, n))
        D = 0.5 * (D + D.T)
        tau = 1e-9
    b = fk.JKBuilder(bas, tau)
    Dt = _dev(torch, D)
    J, none = b.build(Dt, parts="j")
    none2, K = b.build(Dt, parts="k")
    torch.cuda.synchronize()
    assert none is None and none2 is None and fk.fock_stream_status() == 0
    Jo, _ = oracle.jk(bas, D, tau, oracle.SCREEN_DENSITY_J)
    _, Ko = oracle.jk(bas, D, tau, oracle.SCREEN_DENSITY_K)
    ej = float(np.abs(J.cpu().numpy() - Jo).max())
    ek = float(np.abs(K.cpu().numpy() - Ko).max())
    print(f"{case}: J-only max|dJ|={ej:.2e}, K-only max|dK|={ek:.2e}")
    assert ej <= TOL and ek <= TOL, (ej, ek)
    b.close()


@pytest.mark.parametrize("config,kw", [(1, {}), (2, {"waters": 16})])
def test_decay_fit_and_radii_match_oracle(env, config, kw):
    torch, fk = env
    p = molgen.problem(config, **kw)
    b = fk.JKBuilder(p.basis, p.tau, fk.make_opts(k_mode=1))
    H, L, R, Gs = b.decay_bound(_dev(torch, p.D))
    Dsh = decay.shell_block_max(p.basis, p.D)
    Ho, Lo = decay.decay_fit(decay.decay_bins(p.basis, Dsh))
    G, Gp = oracle.schwarz(p.basis)
    Ro, Gso = decay.shell_radii(p.basis, G, Gp, p.tau)
    print(f"config {config}: H={H:.6g} (oracle {Ho:.6g}) Lambda={L:.6g} (oracle {Lo:.6g}) max R={R.max():.3f}")
    assert abs(H - Ho) <= 1e-10 * Ho and abs(L - Lo) <= 1e-10 * abs(Lo)
    assert np.abs(R - Ro).max() <= 1e-12 * max(1.0, Ro.max())
    assert np.abs(Gs - Gso).max() <= 1e-12 * Gso.max()
    b.close()


def test_decay_mode_error_against_exact(env):
    """C20H42, tau* = 5e-6: the decay-bound mode drops only exchange
    contributions; the stated bound is max|dK| <= 1e-4 and
    |tr(D dK)| <= 1e-4 against the exact mode (the paper reports HF energies
    within 1e-5 Eh at this tau*).  J is exact up to quartets whose own J
    bound is below tau."""
    torch, fk = env
    p = molgen.problem(1)
    Dt = _dev(torch, p.D)
    ex = fk.JKBuilder(p.basis, p.tau)
    dc = fk.JKBuilder(p.basis, p.tau, fk.make_opts(k_mode=1, k_thresh=5e-6))
    J0, K0 = ex.build(Dt)
    J1, K1 = dc.build(Dt)
    _, K2 = dc.build(Dt, parts="k")
    torch.cuda.synchronize()
    assert fk.fock_stream_status() == 0
    dK = (K1 - K0).cpu().numpy()
    dK2 = (K2 - K0).cpu().numpy()
    dJ = float((J1 - J0).abs().max())
    tr = abs(float(np.sum(p.D * dK)))
    print(f"C20H42 decay mode: max|dK|={np.abs(dK).max():.2e} (K only {np.abs(dK2).max():.2e}) "
          f"|tr(D dK)|={tr:.2e} max|dJ|={dJ:.2e}")
    assert np.abs(dK).max() <= 1e-4 and np.abs(dK2).max() <= 1e-4 and tr <= 1e-4
    assert dJ <= 1e-8
    ex.close()
    dc.close()


def test_decay_mode_tiny_threshold_keeps_every_schwarz_quartet(env):
    """With tau* far below every contribution the decay-bound test keeps every
    Schwarz-passing quartet: K equals the Schwarz-only oracle K within 1e-10,
    and is at least as close to it as the exact K-only build, which drops the
    quartets whose density-weighted bound is below tau."""
    torch, fk = env
    p = molgen.problem(1, carbons=12)
    Dt = _dev(torch, p.D)
    ex = fk.JKBuilder(p.basis, p.tau)
    dc = fk.JKBuilder(p.basis, p.tau, fk.make_opts(k_mode=1, k_thresh=1e-16))
    _, K0 = ex.build(Dt, parts="k")
    _, K1 = dc.build(Dt, parts="k")
    torch.cuda.synchronize()
    _, Ks = oracle.jk(p.basis, p.D, p.tau, oracle.SCREEN_SCHWARZ)
    e1 = float(np.abs(K1.cpu().numpy() - Ks).max())
    e0 = float(np.abs(K0.cpu().numpy() - Ks).max())
    print(f"C12H26: decay mode (tau* 1e-16) vs Schwarz-only K {e1:.2e}; exact mode {e0:.2e}")
    assert e1 <= 1e-10 and e1 <= e0 + 1e-12
    ex.close()
    dc.close()


def test_decay_mode_rejected_by_batched_build(env):
    torch, fk = env
    p = molgen.problem(0)
    b = fk.JKBuilder(p.basis, p.tau, fk.make_opts(k_mode=1))
    Dt = _dev(torch, p.D)
    J, K = torch.empty_like(Dt), torch.empty_like(Dt)
    with pytest.raises(fk.FockError):
        fk.fock_build_jk_batched([b.handle], [Dt], p.tau, [J], [K])
    b.close()
