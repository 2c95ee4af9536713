"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
independent of the oracle's own code paths (closed forms, quadrature,
identities, brute force).  None of these needs a GPU."""
import math

import numpy as np
import pytest

import molgen
import oracle


def cart_list(l):
    return [(x, y, l - x - y) for x in range(l, -1, -1) for y in range(l - x, -1, -1)]


# --------------------------------------------------------------------------
# Boys function (Eq. boys-fn-def)
# --------------------------------------------------------------------------

def test_boys_at_zero():
    F = oracle.boys(18, 0.0)
    assert np.allclose(F, [1.0 / (2 * m + 1) for m in range(19)], rtol=1e-15, atol=0)


def test_boys_f0_erf_closed_form():
    for T in np.concatenate([np.linspace(1e-6, 2, 17), np.linspace(2, 120, 41)]):
        ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        assert abs(oracle.boys(0, T)[0] - ref) <= 2e-15 * ref


def test_boys_gauss_legendre_quadrature(rng):
    """int_0^1 t^{2m} exp(-T t^2) dt by composite Gauss-Legendre (8 panels x 32
    points, 256 nodes; a single 200-node rule carries ~1e-13 node errors)."""
    x, w = np.polynomial.legendre.leggauss(32)
    t = np.concatenate([(k + 0.5 * (x + 1.0)) / 8 for k in range(8)])
    w = np.concatenate([w / 16] * 8)
    for _ in range(400):
        m = int(rng.integers(0, 19))
        T = float(rng.choice([rng.uniform(0, 1), rng.uniform(1, 40), rng.uniform(40, 120)]))
        ref = np.sum(w * t ** (2 * m) * np.exp(-T * t * t))
        F = oracle.boys(m, T)[m]
        assert abs(F - ref) <= 1e-13 * ref, (m, T, F, ref)


def test_boys_downward_recurrence_identity(rng):
    for _ in range(100):
        T = float(rng.uniform(0, 100))
        F = oracle.boys(12, T)
        for m in range(12):
            lhs = (2 * m + 1) * F[m]
            rhs = 2 * T * F[m + 1] + math.exp(-T)
            assert abs(lhs - rhs) <= 1e-14 * lhs


# --------------------------------------------------------------------------
# normalisation (Sec. 2.1): every Cartesian function has unit self-overlap
# --------------------------------------------------------------------------

def test_overlap_diagonal_is_one():
    p = molgen.problem(0)
    S = oracle.overlap(p.basis)
    assert np.abs(np.diag(S) - 1).max() < 1e-14
    assert np.abs(S - S.T).max() < 1e-14
    # Gram matrix of linearly independent functions is positive definite
    assert np.linalg.eigvalsh(S).min() > 0


def test_overlap_two_s_closed_form(rng):
    """<s_A|s_B> = (4ab/(a+b)^2)^(3/4) exp(-ab/(a+b) R^2) for normalised primitives."""
    for _ in range(20):
        a, b = rng.uniform(0.1, 20, 2)
        A, B = rng.uniform(-2, 2, (2, 3))
        bas = molgen.single_shell_basis([(0, A, [a], [1.0]), (0, B, [b], [1.0])])
        S = oracle.overlap(bas)
        ref = (4 * a * b / (a + b) ** 2) ** 0.75 * math.exp(-a * b / (a + b) * np.sum((A - B) ** 2))
        assert abs(S[0, 1] - ref) <= 1e-14


# --------------------------------------------------------------------------
# ERIs
# --------------------------------------------------------------------------

def test_ssss_closed_form(rng):
    """[ss|ss] = 2 pi^{5/2} / (p q sqrt(p+q)) K_AB K_CD F_0(T) (unit primitives)."""
    for _ in range(200):
        a, b, c, d = rng.uniform(0.05, 50, 4)
        A, B, C, D = rng.uniform(-3, 3, (4, 3))
        p, q = a + b, c + d
        P, Q = (a * A + b * B) / p, (c * C + d * D) / q
        T = p * q / (p + q) * np.sum((P - Q) ** 2)
        F0 = 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        ref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * math.exp(
            -a * b / p * np.sum((A - B) ** 2) - c * d / q * np.sum((C - D) ** 2)) * F0
        v = oracle.prim_eri(0, 0, 0, 0, a, A, b, B, c, C, d, D)[0, 0, 0, 0]
        assert abs(v - ref) <= 1e-13 * abs(ref) + 1e-250, (v, ref)


def test_single_s_self_repulsion():
    """A normalised s Gaussian of exponent a: (ss|ss) = 2 sqrt(a/pi); a one-shell
    basis then has J_00 = K_00 = (ss|ss) D_00."""
    for a in (0.3, 1.0, 7.5):
        bas = molgen.single_shell_basis([(0, [0.1, -0.2, 0.3], [a], [1.0])])
        v = oracle.shell_eri(bas, 0, 0, 0, 0)[0, 0, 0, 0]
        assert abs(v - 2 * math.sqrt(a / math.pi)) < 1e-14
        D = np.array([[0.7]])
        J, K = oracle.jk(bas, D, tau=0.0, mode=oracle.SCREEN_NONE, eps_prune=0.0)
        assert abs(J[0, 0] - v * 0.7) < 1e-14 and abs(K[0, 0] - v * 0.7) < 1e-14


def _quadrature_eri(la, lb, lc, ld, a, A, b, B, c, C, d, D, nt=400):
    """Brute force: 1/r12 = 2/sqrt(pi) int_0^inf exp(-t^2 r12^2) dt; for fixed t
    the 6-D integral factorises into three 2-D Gaussian moments, done exactly
    with 2-D Gauss-Hermite in the eigenbasis of the quadratic form."""
    p, q = a + b, c + d
    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
    pref = math.exp(-a * b / p * np.sum((A - B) ** 2) - c * d / q * np.sum((C - D) ** 2))
    gx, gw = np.polynomial.hermite.hermgauss(12)
    Y1, Y2 = np.meshgrid(gx, gx, indexing="ij")
    W = np.outer(gw, gw)
    scale = math.sqrt(p * q / (p + q))
    s, ws = np.polynomial.legendre.leggauss(nt)
    s = 0.5 * (s + 1)
    ws = 0.5 * ws
    ts = scale * s / (1 - s)
    dts = scale / (1 - s) ** 2
    la_c, lb_c, lc_c, ld_c = (np.array(cart_list(l)) for l in (la, lb, lc, ld))
    # component exponents of every (ia, ib, ic, id) combination, per axis
    ua = la_c[:, None, None, None, :]
    ub = lb_c[None, :, None, None, :]
    uc = lc_c[None, None, :, None, :]
    ud = ld_c[None, None, None, :, :]
    shape = (len(la_c), len(lb_c), len(lc_c), len(ld_c))
    idx = [np.broadcast_to(x, shape + (3,)) for x in (ua, ub, uc, ud)]
    acc = np.zeros(shape)
    for t, wt, dt in zip(ts, ws, dts):
        val = np.ones(shape)
        for ax in range(3):
            # quadratic form p(x1-P)^2 + q(x2-Q)^2 + t^2 (x1-x2)^2
            M = np.array([[p + t * t, -t * t], [-t * t, q + t * t]])
            rhs = np.array([p * P[ax], q * Q[ax]])
            m0 = np.linalg.solve(M, rhs)
            c0 = p * P[ax] ** 2 + q * Q[ax] ** 2 - rhs @ m0
            lam, V = np.linalg.eigh(M)
            X1 = m0[0] + V[0, 0] * Y1 / math.sqrt(lam[0]) + V[0, 1] * Y2 / math.sqrt(lam[1])
            X2 = m0[1] + V[1, 0] * Y1 / math.sqrt(lam[0]) + V[1, 1] * Y2 / math.sqrt(lam[1])
            jac = math.exp(-c0) / math.sqrt(lam[0] * lam[1])
            # moments[i, j, k, m] = int int (x1-A)^i (x1-B)^j (x2-C)^k (x2-D)^m e^{-Q}
            pa = (X1 - A[ax])[None] ** np.arange(la + 1)[:, None, None]
            pb = (X1 - B[ax])[None] ** np.arange(lb + 1)[:, None, None]
            pc = (X2 - C[ax])[None] ** np.arange(lc + 1)[:, None, None]
            pd = (X2 - D[ax])[None] ** np.arange(ld + 1)[:, None, None]
            mom = jac * np.einsum("xy,ixy,jxy,kxy,mxy->ijkm", W, pa, pb, pc, pd)
            val = val * mom[idx[0][..., ax], idx[1][..., ax], idx[2][..., ax], idx[3][..., ax]]
        acc += wt * dt * val
    return pref * 2 / math.sqrt(math.pi) * acc


@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0), (1, 1, 1, 1),
                                (2, 0, 1, 0), (2, 1, 2, 0), (2, 2, 1, 1), (2, 2, 2, 2), (3, 0, 1, 0),
                                (3, 1, 2, 0), (3, 3, 0, 0), (3, 3, 2, 2), (3, 3, 3, 3)])
def test_eri_brute_force_quadrature(ls, rng):
    la, lb, lc, ld = ls
    a, b, c, d = rng.uniform(0.3, 3.0, 4)
    A, B, C, D = rng.uniform(-1.0, 1.0, (4, 3))
    ref = _quadrature_eri(la, lb, lc, ld, a, A, b, B, c, C, d, D)
    val = oracle.prim_eri(la, lb, lc, ld, a, A, b, B, c, C, d, D)
    err = np.abs(val - ref).max() / np.abs(ref).max()
    assert err < 1e-11, err


def test_centre_derivative_identity(rng):
    """d/dA_x [a b|c d] = 2 alpha [a+1_x b|c d] - a_x [a-1_x b|c d] (Sec. 2.1)."""
    for la, lb, lc, ld in [(0, 1, 1, 0), (1, 1, 0, 1), (2, 1, 1, 0), (2, 2, 1, 1), (3, 1, 2, 0), (3, 2, 3, 3)]:
        a, b, c, d = rng.uniform(0.3, 2.0, 4)
        A, B, C, D = rng.uniform(-1.0, 1.0, (4, 3))
        up = oracle.prim_eri(la + 1, lb, lc, ld, a, A, b, B, c, C, d, D)
        dn = oracle.prim_eri(la - 1, lb, lc, ld, a, A, b, B, c, C, d, D) if la > 0 else None
        h = 1e-3
        for ax in range(3):
            def f(delta):
                A2 = A.copy()
                A2[ax] += delta
                return oracle.prim_eri(la, lb, lc, ld, a, A2, b, B, c, C, d, D)
            fd = (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)
            comps = cart_list(la)
            up_c, dn_c = cart_list(la + 1), cart_list(la - 1) if la > 0 else []
            for ia, u in enumerate(comps):
                uu = list(u)
                uu[ax] += 1
                ana = 2 * a * up[up_c.index(tuple(uu))]
                if u[ax] > 0:
                    ud = list(u)
                    ud[ax] -= 1
                    ana = ana - u[ax] * dn[dn_c.index(tuple(ud))]
                scale = max(np.abs(ana).max(), 1e-3)
                assert np.abs(fd[ia] - ana).max() <= 1e-7 * scale, (ls, ax, ia)


def test_eightfold_symmetry(rng):
    bas = molgen.random_shells(rng, [0, 1, 2, 3, 1, 2], spread=1.2)
    for a, b, c, d in [(1, 2, 3, 4), (3, 0, 5, 2), (2, 2, 1, 5), (3, 3, 3, 3), (5, 4, 2, 1)]:
        e = oracle.shell_eri(bas, a, b, c, d)
        ref = np.abs(e).max()
        perms = [((b, a, c, d), (1, 0, 2, 3)), ((a, b, d, c), (0, 1, 3, 2)), ((b, a, d, c), (1, 0, 3, 2)),
                 ((c, d, a, b), (2, 3, 0, 1)), ((d, c, a, b), (3, 2, 0, 1)), ((c, d, b, a), (2, 3, 1, 0)),
                 ((d, c, b, a), (3, 2, 1, 0))]
        for (s0, s1, s2, s3), axes in perms:
            e2 = oracle.shell_eri(bas, s0, s1, s2, s3)
            # e2[i0,i1,i2,i3] with i_k the component of shell s_k; map back
            back = np.transpose(e2, np.argsort(axes))
            assert np.abs(back - e).max() <= 5e-14 * ref


def test_schwarz_inequality(rng):
    bas = molgen.random_shells(rng, [0, 1, 2, 3, 0, 1, 2], spread=2.0)
    G, Gp = oracle.schwarz(bas)
    ns = len(bas["l"])
    for _ in range(40):
        a, b, c, d = rng.integers(0, ns, 4)
        e = oracle.shell_eri(bas, a, b, c, d)
        assert np.abs(e).max() <= G[a, b] * G[c, d] * (1 + 1e-12)
    # diagonal element (mn|mn) = G^2 for the maximising pair
    for a, b in [(0, 1), (2, 3), (4, 6)]:
        e = oracle.shell_eri(bas, a, b, a, b)
        n = e.shape[0] * e.shape[1]
        diag = np.diag(e.reshape(n, n))
        assert abs(math.sqrt(diag.max()) - G[a, b]) <= 1e-13 * G[a, b]
        assert G[a, b] == G[b, a]


def test_translation_invariance(rng):
    bas = molgen.random_shells(rng, [1, 2, 0, 3, 2], spread=1.5)
    shift = rng.uniform(-5, 5, 3)
    bas2 = dict(bas)
    bas2["center"] = bas["center"] + shift
    for q in [(0, 1, 2, 3), (4, 3, 1, 0), (1, 1, 4, 2)]:
        e1, e2 = oracle.shell_eri(bas, *q), oracle.shell_eri(bas2, *q)
        assert np.abs(e1 - e2).max() <= 1e-13 * np.abs(e1).max()


def test_rotation_covariance_sp(rng):
    """s functions are invariant and p functions rotate as vectors, so J and K
    of the rotated molecule equal T J T^T for the rotated density T D T^T."""
    bas = molgen.random_shells(rng, [0, 1, 1, 0, 1], spread=1.5)
    Rm = molgen.random_rotation(rng)
    bas2 = dict(bas)
    bas2["center"] = bas["center"] @ Rm.T
    n = oracle.nbf(bas)
    T = np.zeros((n, n))
    o = 0
    for l in bas["l"]:
        if l == 0:
            T[o, o] = 1.0
        else:
            T[o:o + 3, o:o + 3] = Rm
        o += oracle.ncart(int(l))
    D = rng.uniform(-1, 1, (n, n))
    D = D + D.T
    J, K = oracle.jk(bas, D, mode=oracle.SCREEN_NONE, eps_prune=0.0)
    J2, K2 = oracle.jk(bas2, T @ D @ T.T, mode=oracle.SCREEN_NONE, eps_prune=0.0)
    assert np.abs(J2 - T @ J @ T.T).max() < 1e-12
    assert np.abs(K2 - T @ K @ T.T).max() < 1e-12


# --------------------------------------------------------------------------
# J / K (Eq. fock_build) properties
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_case():
    r = np.random.Generator(np.random.PCG64(77))
    bas = molgen.random_shells(r, [0, 1, 2, 0, 3, 1], spread=1.5)
    n = oracle.nbf(bas)
    D = r.uniform(-1, 1, (n, n))
    return bas, D + D.T


def test_jk_symmetric_linear_psd(small_case, rng):
    bas, D = small_case
    J, K = oracle.jk(bas, D, mode=oracle.SCREEN_NONE, eps_prune=0.0)
    assert np.abs(J - J.T).max() < 1e-13 and np.abs(K - K.T).max() < 1e-13
    D2 = rng.uniform(-1, 1, D.shape)
    D2 = D2 + D2.T
    J2, K2 = oracle.jk(bas, D2, mode=oracle.SCREEN_NONE, eps_prune=0.0)
    J3, K3 = oracle.jk(bas, D + 2 * D2, mode=oracle.SCREEN_NONE, eps_prune=0.0)
    assert np.abs(J3 - (J + 2 * J2)).max() < 1e-12 and np.abs(K3 - (K + 2 * K2)).max() < 1e-12
    # Coulomb and exchange energies of a symmetric D are non-negative
    assert np.sum(D * J) > 0 and np.sum(D * K) > 0
    assert np.sum(D2 * J2) > 0 and np.sum(D2 * K2) > 0


def test_jk_symmetric_scatter_matches_all_quartets(small_case):
    bas, D = small_case
    for mode, tau, eps in [(oracle.SCREEN_NONE, 0.0, 0.0), (oracle.SCREEN_DENSITY, 1e-3, 1e-3)]:
        J1, K1 = oracle.jk(bas, D, tau=tau, mode=mode, eps_prune=eps, symmetric=True)
        J2, K2 = oracle.jk(bas, D, tau=tau, mode=mode, eps_prune=eps, symmetric=False)
        assert np.abs(J1 - J2).max() < 1e-12 and np.abs(K1 - K2).max() < 1e-12


def test_probe_density_recovers_eris(small_case):
    """D = e_ls + e_sl gives J_mn = 2 (mn|ls) and K_mn = (ml|ns) + (ms|nl)."""
    bas, _ = small_case
    n = oracle.nbf(bas)
    offs = np.concatenate([[0], np.cumsum([oracle.ncart(int(l)) for l in bas["l"]])])
    a, b, c, d = 1, 2, 4, 5
    e = oracle.shell_eri(bas, a, b, c, d)
    lam, sig = offs[c] + 1, offs[d] + 2
    D = np.zeros((n, n))
    D[lam, sig] = D[sig, lam] = 1.0
    J, K = oracle.jk(bas, D, mode=oracle.SCREEN_NONE, eps_prune=0.0)
    blkJ = J[offs[a]:offs[a + 1], offs[b]:offs[b + 1]]
    assert np.abs(blkJ - 2 * e[:, :, 1, 2]).max() < 1e-13
    # K_mn = (m lam | n sig) + (m sig | n lam)
    e2 = oracle.shell_eri(bas, a, c, b, d)
    e3 = oracle.shell_eri(bas, a, d, b, c)
    blkK = K[offs[a]:offs[a + 1], offs[b]:offs[b + 1]]
    assert np.abs(blkK - (e2[:, 1, :, 2] + e3[:, 2, :, 1])).max() < 1e-13


def test_blocks_match_full(small_case):
    bas, D = small_case
    J, K = oracle.jk(bas, D, tau=1e-4, mode=oracle.SCREEN_DENSITY, eps_prune=1e-3)
    offs = np.concatenate([[0], np.cumsum([oracle.ncart(int(l)) for l in bas["l"]])])
    pairs = [(0, 0), (2, 1), (4, 4), (1, 5), (5, 3)]
    Jb, Kb = oracle.jk_blocks(bas, D, pairs, tau=1e-4, mode=oracle.SCREEN_DENSITY, eps_prune=1e-3)
    for (a, b), jb, kb in zip(pairs, Jb, Kb):
        assert np.abs(J[offs[a]:offs[a + 1], offs[b]:offs[b + 1]] - jb).max() < 1e-13
        assert np.abs(K[offs[a]:offs[a + 1], offs[b]:offs[b + 1]] - kb).max() < 1e-13


def test_screening_error_bounded():
    """Each skipped contracted quartet moves a J or K element by at most
    (number of its terms) x G_ab G_cd Dmax < 100 tau; the crude rigorous bound
    below sums that over every quartet that can feed one element."""
    r = np.random.Generator(np.random.PCG64(5))
    bas = molgen.random_shells(r, [0, 1, 2, 0, 1, 2, 0, 1], spread=5.0)
    n = oracle.nbf(bas)
    D = r.uniform(-1, 1, (n, n))
    D = D + D.T
    tau = 1e-4
    J0, K0 = oracle.jk(bas, D, mode=oracle.SCREEN_NONE, eps_prune=0.0)
    J2, K2 = oracle.jk(bas, D, tau=tau, mode=oracle.SCREEN_DENSITY, eps_prune=0.0)
    ns = len(bas["l"])
    bound = 8 * ns * ns * 36 * tau
    assert np.abs(J0 - J2).max() <= bound and np.abs(K0 - K2).max() <= bound
    assert np.abs(J0 - J2).max() > 0 or np.abs(K0 - K2).max() > 0  # something was screened
    cnt = oracle.count(bas, D, tau)
    assert cnt["quartets_density"] < ns * (ns + 1) // 2 * (ns * (ns + 1) // 2 + 1) // 2


def test_count_matches_brute_force():
    p = molgen.problem(0)
    G, _ = oracle.schwarz(p.basis)
    ls = p.basis["l"]
    ns = len(ls)
    q = e = 0
    for a in range(ns):
        for b in range(a + 1):
            for c in range(a + 1):
                for d in range(c + 1):
                    if (c, d) > (a, b):
                        continue
                    if G[a, b] * G[c, d] >= p.tau:
                        q += 1
                        e += np.prod([oracle.ncart(int(ls[s])) for s in (a, b, c, d)])
    cnt = oracle.count(p.basis, p.D, p.tau)
    assert cnt["quartets_schwarz"] == q and cnt["eris_schwarz"] == e


# --------------------------------------------------------------------------
# one-electron integrals (core Hamiltonian h = T + V, Sec. 2.2)
# --------------------------------------------------------------------------

def test_one_electron_single_gaussian_closed_forms():
    """Normalised Gaussian r^l exp(-a r^2) on a nucleus of charge Z:
    T = (2l+3) a / 2 and <1/r> = 2^(l+1) l! sqrt(2a) / ((2l+1)!! sqrt(pi))."""
    C = np.array([0.3, -0.2, 0.1])
    for a in (0.3, 2.0, 11.0):
        for l, comp in ((0, 0), (1, 0), (1, 2)):
            bas = molgen.single_shell_basis([(l, C, [a], [1.0])])
            T = oracle.kinetic(bas)
            V = oracle.nuclear(bas, [3.0], [C])
            dfact = 1 if l == 0 else 3
            r1 = 2 ** (l + 1) * math.factorial(l) * math.sqrt(2 * a) / (dfact * math.sqrt(math.pi))
            assert abs(T[comp, comp] - (2 * l + 3) * a / 2) < 1e-13 * a
            assert abs(V[comp, comp] + 3.0 * r1) < 1e-13 * r1


def test_one_electron_two_s_closed_forms(rng):
    """T_ab = mu (3 - 2 mu R^2) S_ab; V_ab = -Z 2pi/p K_AB N_a N_b F_0(p |PC|^2)."""
    for _ in range(20):
        a, b = rng.uniform(0.2, 6, 2)
        A, B, Cn = rng.uniform(-1.5, 1.5, (3, 3))
        bas = molgen.single_shell_basis([(0, A, [a], [1.0]), (0, B, [b], [1.0])])
        S = oracle.overlap(bas)
        T = oracle.kinetic(bas)
        V = oracle.nuclear(bas, [1.7], [Cn])
        mu, p = a * b / (a + b), a + b
        R2 = np.sum((A - B) ** 2)
        assert abs(T[0, 1] - mu * (3 - 2 * mu * R2) * S[0, 1]) < 1e-13
        P = (a * A + b * B) / p
        Tn = p * np.sum((P - Cn) ** 2)
        F0 = 1.0 if Tn == 0 else 0.5 * math.sqrt(math.pi / Tn) * math.erf(math.sqrt(Tn))
        Na, Nb = (2 * a / math.pi) ** 0.75, (2 * b / math.pi) ** 0.75
        ref = -1.7 * 2 * math.pi / p * math.exp(-mu * R2) * Na * Nb * F0
        assert abs(V[0, 1] - ref) < 1e-13 * abs(ref)


def test_one_electron_invariances(rng):
    bas = molgen.random_shells(rng, [0, 1, 2, 3, 1], spread=1.5)
    Zs = np.array([1.0, 6.0, 8.0])
    at = rng.uniform(-2, 2, (3, 3))
    shift = rng.uniform(-4, 4, 3)
    bas2 = dict(bas)
    bas2["center"] = bas["center"] + shift
    T1, T2 = oracle.kinetic(bas), oracle.kinetic(bas2)
    V1, V2 = oracle.nuclear(bas, Zs, at), oracle.nuclear(bas2, Zs, at + shift)
    assert np.abs(T1 - T2).max() < 1e-12 and np.abs(V1 - V2).max() < 1e-11
    assert np.abs(T1 - T1.T).max() < 1e-12 and np.abs(V1 - V1.T).max() < 1e-11
    # the kinetic energy operator is positive definite on independent functions
    assert np.linalg.eigvalsh(T1).min() > 0


def _dfact(n):
    return 1 if n <= 0 else n * _dfact(n - 2)


def _one_electron_quadrature(la, a, A, lb, b, B, Zs, Cs, nt=400):
    """Brute force S, T, V between two primitive Cartesian shells, normalised
    to unit self-overlap, without the Boys function or any recurrence.
    Per axis the 1-D integrals of polynomial x Gaussian are exact by
    Gauss-Hermite after completing the square; T applies the second derivative
    to the ket factor (-1/2 nabla^2); 1/|r-C| = 2/sqrt(pi) int_0^inf
    exp(-t^2 |r-C|^2) dt with the t integral by mapped Gauss-Legendre."""
    gx, gw = np.polynomial.hermite.hermgauss(16)

    def line(i, j, ax, t2=0.0, c=0.0, deriv=False):
        g = a + b + t2
        x0 = (a * A[ax] + b * B[ax] + t2 * c) / g
        k0 = a * A[ax] ** 2 + b * B[ax] ** 2 + t2 * c * c - g * x0 * x0
        x = x0 + gx / math.sqrt(g)
        xa, xb = x - A[ax], x - B[ax]
        if deriv:  # d^2/dx^2 of (x-B)^j exp(-b (x-B)^2), Gaussian factor kept apart
            fb = 4 * b * b * xb ** (j + 2) - 2 * b * (2 * j + 1) * xb ** j
            if j >= 2:
                fb = fb + j * (j - 1) * xb ** (j - 2)
        else:
            fb = xb ** j
        return math.exp(-k0) / math.sqrt(g) * np.sum(gw * xa ** i * fb)

    ca, cb = cart_list(la), cart_list(lb)

    def norm(l, e, X, u):
        g = 2 * e
        return math.sqrt(np.prod([np.sum(gw * (gx / math.sqrt(g)) ** (2 * u[k])) / math.sqrt(g) for k in range(3)]))

    na = [norm(la, a, A, u) for u in ca]
    nb = [norm(lb, b, B, v) for v in cb]
    S = np.zeros((len(ca), len(cb)))
    T = np.zeros_like(S)
    V = np.zeros_like(S)
    s, ws = np.polynomial.legendre.leggauss(nt)
    s = 0.5 * (s + 1)
    ws = 0.5 * ws
    scale = math.sqrt(a + b)
    ts, dts = scale * s / (1 - s), scale / (1 - s) ** 2
    for i, u in enumerate(ca):
        for j, v in enumerate(cb):
            o = [line(u[k], v[k], k) for k in range(3)]
            d2 = [line(u[k], v[k], k, deriv=True) for k in range(3)]
            S[i, j] = np.prod(o)
            T[i, j] = -0.5 * (d2[0] * o[1] * o[2] + o[0] * d2[1] * o[2] + o[0] * o[1] * d2[2])
            acc = 0.0
            for Z, C in zip(Zs, Cs):
                f = [np.prod([line(u[k], v[k], k, t * t, C[k]) for k in range(3)]) for t in ts]
                acc -= Z * 2 / math.sqrt(math.pi) * np.sum(ws * dts * np.array(f))
            V[i, j] = acc
            S[i, j] /= na[i] * nb[j]
            T[i, j] /= na[i] * nb[j]
            V[i, j] /= na[i] * nb[j]
    return S, T, V


@pytest.mark.parametrize("la,lb", [(2, 0), (2, 1), (2, 2), (3, 1), (3, 2), (3, 3)])
def test_one_electron_brute_force_quadrature(la, lb, rng):
    """S, T, V of d and f shells (h = T + V, Sec. 2.2) against quadrature that
    shares no step with the oracle's Obara-Saika recurrences."""
    a, b = rng.uniform(0.3, 3.0, 2)
    A, B = rng.uniform(-1.0, 1.0, (2, 3))
    Zs = [1.0, 6.0]
    Cs = [rng.uniform(-1.5, 1.5, 3), rng.uniform(-1.5, 1.5, 3)]
    Sq, Tq, Vq = _one_electron_quadrature(la, a, A, lb, b, B, Zs, Cs)
    bas = molgen.single_shell_basis([(la, A, [a], [1.0]), (lb, B, [b], [1.0])])
    na = oracle.ncart(la)
    S = oracle.overlap(bas)[:na, na:]
    T = oracle.kinetic(bas)[:na, na:]
    V = oracle.nuclear(bas, Zs, Cs)[:na, na:]
    for ref, val in ((Sq, S), (Tq, T), (Vq, V)):
        assert np.abs(val - ref).max() <= 1e-11 * np.abs(ref).max(), np.abs(val - ref).max()


def test_one_electron_harmonic_d_f_closed_forms():
    """xy, xz, yz and xyz times exp(-a r^2) are pure solid harmonics (l = 2, 3):
    on a nucleus of charge Z, T = (2l+3) a / 2 and
    <1/r> = 2^(l+1) l! sqrt(2a) / ((2l+1)!! sqrt(pi))."""
    C = np.array([-0.4, 0.25, 0.6])
    for a in (0.3, 2.0, 11.0):
        for l, comps in ((2, (1, 2, 4)), (3, (4,))):
            bas = molgen.single_shell_basis([(l, C, [a], [1.0])])
            T = oracle.kinetic(bas)
            V = oracle.nuclear(bas, [2.5], [C])
            r1 = 2 ** (l + 1) * math.factorial(l) * math.sqrt(2 * a) / (_dfact(2 * l + 1) * math.sqrt(math.pi))
            for c in comps:
                assert abs(T[c, c] - (2 * l + 3) * a / 2) < 1e-13 * a
                assert abs(V[c, c] + 2.5 * r1) < 1e-13 * r1


def _rotation_matrix_cart(ls, Rm):
    """M with g_mu = sum_k M[mu, k] phi'_k: a normalised Cartesian function of
    the original molecule, rotated by Rm, expanded in the normalised Cartesian
    functions at the rotated centre.  x^u y^v z^w becomes the product of the
    rotated coordinates (Rm^T s)_i; each monomial's unit-norm factor is
    proportional to 1 / sqrt((2u-1)!! (2v-1)!! (2w-1)!!) within a shell."""
    blocks = []
    for l in ls:
        comps = cart_list(int(l))
        pos = {c: i for i, c in enumerate(comps)}
        nf = [1.0 / math.sqrt(_dfact(2 * c[0] - 1) * _dfact(2 * c[1] - 1) * _dfact(2 * c[2] - 1)) for c in comps]
        Mb = np.zeros((len(comps), len(comps)))
        for i, u in enumerate(comps):
            poly = {(0, 0, 0): 1.0}
            for ax in range(3):
                for _ in range(u[ax]):
                    nxt = {}
                    for e, cf in poly.items():
                        for k in range(3):  # (Rm^T s)_ax = sum_k Rm[k, ax] s_k
                            e2 = list(e)
                            e2[k] += 1
                            nxt[tuple(e2)] = nxt.get(tuple(e2), 0.0) + cf * Rm[k, ax]
                    poly = nxt
            for e, cf in poly.items():
                Mb[i, pos[e]] += nf[i] * cf / nf[pos[e]]
        blocks.append(Mb)
    n = sum(b.shape[0] for b in blocks)
    M = np.zeros((n, n))
    o = 0
    for b in blocks:
        M[o:o + b.shape[0], o:o + b.shape[0]] = b
        o += b.shape[0]
    return M


def test_rotation_covariance_spdf(rng):
    """1/r12 and the kinetic and nuclear operators are rotation invariant, so
    for the molecule rotated by Rm, (mn|ls) = sum M M M M (ab|cd)' and
    J(D) = M J'(M^T D M) M^T, K likewise, S = M S' M^T, etc. (Sec. 2.2
    integrals over Cartesian d and f functions)."""
    ls = [0, 1, 2, 3, 2, 1]
    bas = molgen.random_shells(rng, ls, spread=1.4, kmax=2)
    Rm = molgen.random_rotation(rng)
    bas2 = dict(bas)
    bas2["center"] = bas["center"] @ Rm.T
    M = _rotation_matrix_cart(bas["l"], Rm)
    n = oracle.nbf(bas)
    D = rng.uniform(-1, 1, (n, n))
    D = D + D.T
    J, K = oracle.jk(bas, D, mode=oracle.SCREEN_NONE, eps_prune=0.0)
    J2, K2 = oracle.jk(bas2, M.T @ D @ M, mode=oracle.SCREEN_NONE, eps_prune=0.0)
    assert np.abs(M @ J2 @ M.T - J).max() < 1e-11 * np.abs(J).max()
    assert np.abs(M @ K2 @ M.T - K).max() < 1e-11 * np.abs(K).max()
    Zs = np.array([1.0, 8.0, 6.0])
    at = rng.uniform(-2, 2, (3, 3))
    for f1, f2 in ((oracle.overlap(bas), oracle.overlap(bas2)), (oracle.kinetic(bas), oracle.kinetic(bas2)),
                   (oracle.nuclear(bas, Zs, at), oracle.nuclear(bas2, Zs, at @ Rm.T))):
        assert np.abs(M @ f2 @ M.T - f1).max() < 1e-12 * np.abs(f1).max()


# --------------------------------------------------------------------------
# reference MLP of the learned guess: analytic gradient vs finite differences
# --------------------------------------------------------------------------

def test_mlp_reference_gradient_finite_differences(rng):
    from oracle import mlp_ref
    nin, H, nout, B = 7, 9, 5, 11
    n = H * nin + H + H * H + H + nout * H + nout
    p = rng.normal(0, 0.4, n)
    X = rng.normal(0, 1, (B, nin))
    T = rng.normal(0, 1, (B, nout))
    mask = (rng.uniform(0, 1, (B, nout)) > 0.3).astype(float)
    loss, g = mlp_ref.loss_and_grad(p, X, T, mask, mask.sum(), nin, H, nout, weights_bf16=False)
    for k in rng.choice(n, 25, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        lp, _ = mlp_ref.loss_and_grad(pp, X, T, mask, mask.sum(), nin, H, nout, weights_bf16=False)
        lm, _ = mlp_ref.loss_and_grad(pm, X, T, mask, mask.sum(), nin, H, nout, weights_bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_bf16_rounding_reference():
    from oracle import mlp_ref
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0, 1e-3], dtype=np.float32)
    r = mlp_ref.bf16_round(x)
    # bfloat16 keeps 8 significant bits: relative rounding error <= 2^-9
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8)
    assert r[0] == 1.0 and r[1] == 1.0  # 1 + 2^-8 is a tie that rounds to even


def test_primitive_quartet_screening_brute_force():
    """The primitive-level rules, written out independently over s shells
    from primitive integrals (pinned above by quadrature) and normalised
    coefficients (pinned by the overlap diagonal): a primitive pair [ab] is
    dropped iff G_[ab] Gmax < tau eps, and inside a contracted quartet that
    passes the six-block test a primitive quartet is skipped iff
    G_[ab] G_[cd] Dmax < tau eps (Sec. 3.2 primitive Cauchy-Schwarz bound at
    the level of primitive integrals, Sec. 3.3)."""
    r = np.random.Generator(np.random.PCG64(41))
    bas = molgen.random_shells(r, [0, 0, 0, 0, 0], spread=2.5, kmax=3)
    ns = len(bas["l"])
    D = r.uniform(-1, 1, (ns, ns))
    D = D + D.T
    cn = oracle.norm_coefs(bas)
    ctr, po, npr, ex = bas["center"].reshape(-1, 3), bas["prim_off"], bas["nprim"], bas["exps"]

    def prims(s):
        return [(ex[po[s] + i], cn[po[s] + i]) for i in range(npr[s])]

    def pe(a, b, c, d, pa, pb, pc, pd):
        (ea, ca), (eb, cb), (ec, cc), (ed, cd) = pa, pb, pc, pd
        return ca * cb * cc * cd * oracle.prim_eri(0, 0, 0, 0, ea, ctr[a], eb, ctr[b], ec, ctr[c], ed, ctr[d])[0, 0, 0, 0]

    Gp = {}
    for a in range(ns):
        for b in range(ns):
            Gp[a, b] = np.array([[np.sqrt(abs(pe(a, b, a, b, pa, pb, pa, pb))) for pb in prims(b)] for pa in prims(a)])
    G = np.array([[np.sqrt(abs(sum(pe(a, b, a, b, pa, pb, pc, pd) for pa in prims(a) for pb in prims(b)
                                   for pc in prims(a) for pd in prims(b)))) for b in range(ns)] for a in range(ns)])
    gmax = G.max()
    Dabs = np.abs(D)
    for tau, eps in ((1e-3, 1e-2), (3e-3, 0.5)):
        thr = tau * eps
        nskip = 0

        def eri(a, b, c, d):
            nonlocal nskip
            g = G[a, b] * G[c, d]
            dm = max(Dabs[a, b], Dabs[c, d], Dabs[a, c], Dabs[a, d], Dabs[b, c], Dabs[b, d])
            if g < tau or g * dm < tau:
                return 0.0
            v = 0.0
            for i, pa in enumerate(prims(a)):
                for j, pb in enumerate(prims(b)):
                    if Gp[a, b][i, j] * gmax < thr:
                        continue
                    for k, pc in enumerate(prims(c)):
                        for m, pd in enumerate(prims(d)):
                            if Gp[c, d][k, m] * gmax < thr:
                                continue
                            if Gp[a, b][i, j] * Gp[c, d][k, m] * dm < thr:
                                nskip += 1
                                continue
                            v += pe(a, b, c, d, pa, pb, pc, pd)
            return v

        Jr = np.zeros((ns, ns))
        Kr = np.zeros((ns, ns))
        for a in range(ns):
            for b in range(ns):
                for c in range(ns):
                    for d in range(ns):
                        Jr[a, b] += eri(a, b, c, d) * D[c, d]
                        Kr[a, b] += eri(a, c, b, d) * D[c, d]
        J, K = oracle.jk(bas, D, tau=tau, mode=oracle.SCREEN_DENSITY, eps_prune=eps)
        assert nskip > 0
        assert np.abs(J - Jr).max() < 1e-12 and np.abs(K - Kr).max() < 1e-12
        J0, K0 = oracle.jk(bas, D, tau=tau, mode=oracle.SCREEN_DENSITY, eps_prune=0.0)
        assert np.abs(J - J0).max() > 0
