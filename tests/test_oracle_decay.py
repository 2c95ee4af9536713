"""Pins of the oracle's density decay bound (Sec. 4.3.1, Eq. density_bound)
and of the J-only / K-only screening modes, on the CPU."""
import math

import numpy as np
import pytest

import molgen
import oracle
from oracle import decay


def _line_basis(xs):
    """One s shell per atom at (x, 0, 0) bohr."""
    return molgen.single_shell_basis([(0, [x, 0.0, 0.0], [0.8], [1.0]) for x in xs])


def test_fit_recovers_exact_exponential():
    """Block maxima lying exactly on H0 exp(-L0 r) at the bin centres: the
    least-squares line is that line, and raising it over each whole bin (far
    edge, half a bin beyond the centre) gives H = H0 exp(L0 / 4)."""
    H0, L0 = 0.8, 0.37
    xs = [0.0] + [0.25 + 0.5 * k for k in range(1, 30, 3)]
    bas = _line_basis(xs)
    ns = len(xs)
    Dsh = np.zeros((ns, ns))
    for b in range(1, ns):
        r = xs[b]
        Dsh[0, b] = Dsh[b, 0] = H0 * math.exp(-L0 * (math.floor(r / 0.5) + 0.5) * 0.5)
    bins = decay.decay_bins(bas, Dsh)
    assert len(bins) == ns - 1
    H, L = decay.decay_fit(bins)
    assert abs(L - L0) < 1e-12 * L0
    assert abs(H - H0 * math.exp(L0 * 0.25)) < 1e-12 * H0


def test_fit_degenerate_cases():
    assert decay.decay_fit({}) == (0.0, 0.0)
    H, L = decay.decay_fit({3: 0.25})
    assert L == 0.0 and abs(H - 0.25) < 1e-15


@pytest.mark.parametrize("config", [1, 2])
def test_bound_holds_for_every_off_atom_element(config):
    """|D_mn| <= H exp(-Lambda |CD|) for every pair of functions on different
    atoms (the elements the fit covers), for the synthetic densities."""
    p = molgen.problem(config, carbons=8, waters=12)
    bas = p.basis
    Dsh = decay.shell_block_max(bas, p.D)
    H, L = decay.decay_fit(decay.decay_bins(bas, Dsh))
    assert L > 0.0
    atom = decay.shell_atoms(bas)
    c = bas["center"]
    ns = len(atom)
    worst = 0.0
    for a in range(ns):
        for b in range(ns):
            if atom[a] == atom[b]:
                continue
            r = np.linalg.norm(c[a] - c[b])
            worst = max(worst, Dsh[a, b] / (H * math.exp(-L * r)))
    assert worst <= 1.0 + 1e-12, worst


def test_radius_triangle_inequality():
    """For kept pairs (a, c) and (b, d): |CD| >= |AB| - R_a - R_b (Sec. 4.3.1)."""
    p = molgen.problem(1, carbons=8)
    bas = p.basis
    G, Gp = oracle.schwarz(bas)
    R, Gs = decay.shell_radii(bas, G, Gp, p.tau)
    pairs = decay.kept_pairs(bas, G, Gp, p.tau)
    c = bas["center"]
    rng = np.random.Generator(np.random.PCG64(5))
    idx = rng.integers(0, len(pairs), (20000, 2))
    for i, j in idx:
        for (a, cc), (b, d) in (((pairs[i][0], pairs[i][1]), (pairs[j][0], pairs[j][1])),
                                ((pairs[i][1], pairs[i][0]), (pairs[j][1], pairs[j][0]))):
            lhs = np.linalg.norm(c[cc] - c[d])
            rhs = np.linalg.norm(c[a] - c[b]) - R[a] - R[b]
            assert lhs >= rhs - 1e-12
    # G_s bounds every kept pair's Schwarz factor on either shell
    for a, b in pairs:
        assert G[a, b] <= Gs[a] and G[a, b] <= Gs[b]


def test_decay_bound_bounds_exchange_contributions():
    """Every exchange contribution |(xz|yw) D_zw| of kept pairs (x z), (y w)
    is at most G_xz G_yw H exp(-Lambda (|XY| - R_x - R_y)) wherever that
    exponent argument is positive (sampled quartets of C24H50, whose length
    exceeds twice the radii R_s of about 19 bohr)."""
    p = molgen.problem(1, carbons=24)
    bas = p.basis
    G, Gp = oracle.schwarz(bas)
    R, _ = decay.shell_radii(bas, G, Gp, p.tau)
    Dsh = decay.shell_block_max(bas, p.D)
    H, L = decay.decay_fit(decay.decay_bins(bas, Dsh))
    pairs = np.array(decay.kept_pairs(bas, G, Gp, p.tau))
    c = bas["center"]
    rng = np.random.Generator(np.random.PCG64(9))
    i, j = rng.integers(0, len(pairs), (2, 200000))
    x, y = pairs[i, 0], pairs[j, 0]
    arg = np.linalg.norm(c[x] - c[y], axis=1) - R[x] - R[y]
    sel = np.flatnonzero(arg > 0.0)[:250]
    assert len(sel) == 250
    for k in sel:
        (x, z), (y, w) = pairs[i[k]], pairs[j[k]]
        bound = G[x, z] * G[y, w] * H * math.exp(-L * arg[k])
        e = oracle.shell_eri(bas, x, z, y, w)
        assert np.abs(e).max() * Dsh[z, w] <= bound * (1 + 1e-12)


def test_j_only_and_k_only_screening_modes():
    """Mode 3 weighs a quartet by D_ab, D_cd only and mode 4 by D_ac, D_ad,
    D_bc, D_bd only: with no screening threshold both equal the unscreened
    build; with one, each part's error stays below the sum of the bounds of
    the quartets that part skipped (at most its count x tau)."""
    bas = molgen.random_shells(np.random.Generator(np.random.PCG64(3)), [0, 1, 2, 0, 1, 0], spread=4.0)
    n = oracle.nbf(bas)
    rng = np.random.Generator(np.random.PCG64(4))
    D = rng.uniform(-1, 1, (n, n))
    D = D + D.T
    J0, K0 = oracle.jk(bas, D, 0.0, oracle.SCREEN_NONE, eps_prune=0.0)
    for mode in (oracle.SCREEN_DENSITY_J, oracle.SCREEN_DENSITY_K):
        J, K = oracle.jk(bas, D, 0.0, mode, eps_prune=0.0)
        assert np.abs(J - J0).max() < 1e-12 and np.abs(K - K0).max() < 1e-12
    tau = 1e-4
    Jj, _ = oracle.jk(bas, D, tau, oracle.SCREEN_DENSITY_J, eps_prune=0.0)
    _, Kk = oracle.jk(bas, D, tau, oracle.SCREEN_DENSITY_K, eps_prune=0.0)
    ns = len(bas["l"])
    nq = ns ** 4
    assert np.abs(Jj - J0).max() <= 8 * nq * tau
    assert np.abs(Kk - K0).max() <= 8 * nq * tau
    # on a density that vanishes outside the diagonal shell blocks, J needs
    # the quartets (ab|cc) and K the quartets (ab|cb): weighting either by the
    # other part's blocks would drop them, so each mode must reproduce its
    # part of the unscreened build
    Db = np.zeros_like(D)
    off = np.concatenate([[0], np.cumsum([oracle.ncart(int(l)) for l in bas["l"]])])
    for s in range(ns):
        Db[off[s]:off[s + 1], off[s]:off[s + 1]] = D[off[s]:off[s + 1], off[s]:off[s + 1]]
    Jf, Kf = oracle.jk(bas, Db, 0.0, oracle.SCREEN_NONE, eps_prune=0.0)
    Jj, _ = oracle.jk(bas, Db, 1e-12, oracle.SCREEN_DENSITY_J, eps_prune=0.0)
    _, Kk = oracle.jk(bas, Db, 1e-12, oracle.SCREEN_DENSITY_K, eps_prune=0.0)
    assert np.abs(Jj - Jf).max() < 1e-12 and np.abs(Kk - Kf).max() < 1e-12
