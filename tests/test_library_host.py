"""Host-side checks of libfock.so that need no GPU: the library loads and
exports every entry point include/fock.h declares, its Boys table and Hermite
coefficients meet the paper's printed facts and independent references, and
argument validation returns the documented status codes."""
import ctypes
import json
import math
import os

import numpy as np

import molgen
import oracle
import paper_2407_21445_gb300 as fk
from paper_2407_21445_gb300 import fock as fb

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")))


def cart_list(l):
    return [(x, y, l - x - y) for x in range(l, -1, -1) for y in range(l - x, -1, -1)]


def test_library_exports_every_declared_symbol():
    names = fb.declared_symbols()
    assert len(names) >= 12
    L = fb.lib()
    for n in names:
        assert hasattr(L, n), n


def test_binding_has_every_entry_point():
    """The Python binding offers each C entry point under its own name."""
    for n in fb.declared_symbols():
        assert callable(getattr(fb, n, None)), n


def test_status_strings():
    for i, name in enumerate(fb.STATUS_NAMES):
        assert fk.fock_status_string(i) == name


def test_boys_table_matches_oracle_and_quadrature(rng):
    info = fk.fock_boys_table_info()
    assert info["h"] == 1 / 16 and info["tmax"] == 64.0
    x, w = np.polynomial.legendre.leggauss(32)
    t = np.concatenate([(k + 0.5 * (x + 1.0)) / 8 for k in range(8)])
    w = np.concatenate([w / 16] * 8)
    Ts = np.concatenate([rng.uniform(0, 64, 300), rng.uniform(64, 500, 50), np.arange(0, 64, 1 / 16)[::7],
                         [0.0, 1e-12, 63.999999, 64.0]])
    for T in Ts:
        F = fk.fock_boys_host(12, T)
        Fo = oracle.boys(12, T)
        assert np.max(np.abs(F - Fo) / Fo) < 5e-15, T
    for T in rng.uniform(0, 80, 40):
        F = fk.fock_boys_host(12, T)
        for m in (0, 5, 12):
            ref = np.sum(w * t ** (2 * m) * np.exp(-T * t * t))
            assert abs(F[m] - ref) <= 1e-13 * ref


def test_hermite_counts_match_paper():
    g = GOLD["hermite_tensor_dd"]
    assert fk.fock_hermite_count(2, 2) == g["nonzero"]
    assert 6 * 6 * (4 + 1) * (4 + 2) * (4 + 3) // 6 == g["dense_elements"]
    # nonzero count = sum over Cartesian pairs of prod (a_i + b_i + 1)
    for la in range(4):
        for lb in range(la + 1):
            n = sum((a[0] + b[0] + 1) * (a[1] + b[1] + 1) * (a[2] + b[2] + 1)
                    for a in cart_list(la) for b in cart_list(lb))
            assert fk.fock_hermite_count(la, lb) == n
    assert GOLD["pp_pp_integrals"]["count"] == len(cart_list(1)) ** 4
    assert GOLD["cartesian_functions_per_shell"]["by_l"] == [len(cart_list(l)) for l in range(4)]


def test_hermite_top_coefficient_and_trivial(rng):
    """E^{ab}_{a+b} = 1/(2 zeta)^{a+b} (Eq. MMD-observation) and E^{00}_0 = 1."""
    e = fk.fock_hermite_e(0, 0, 0.7, [0, 0, 0], 1.3, [0.2, 0.1, -0.3])
    assert e.shape == (1,) and e[0] == 1.0
    for la in range(4):
        for lb in range(la + 1):
            a, b = rng.uniform(0.2, 5, 2)
            A, B = rng.uniform(-1, 1, (2, 3))
            E = fk.fock_hermite_e(la, lb, a, A, b, B)
            z = a + b
            o = 0
            for ca in cart_list(la):
                for cb in cart_list(lb):
                    T = [ca[i] + cb[i] for i in range(3)]
                    n = (T[0] + 1) * (T[1] + 1) * (T[2] + 1)
                    top = E[o + n - 1]  # (t,u,v) = (Tx,Ty,Tz) is last in t-major order
                    assert abs(top - (2 * z) ** (-sum(T))) <= 1e-14 * (2 * z) ** (-sum(T))
                    o += n


def test_hermite_zero_term_is_overlap(rng):
    """<a|b> = E^{ab}_{000} (pi/zeta)^{3/2} K_AB; compared with the oracle's
    Obara-Saika overlap of the same two normalised primitives."""
    for la, lb in [(1, 0), (2, 1), (3, 2), (2, 2), (3, 3)]:
        a, b = rng.uniform(0.3, 3, 2)
        A, B = rng.uniform(-1, 1, (2, 3))
        bas = molgen.single_shell_basis([(la, A, [a], [1.0]), (lb, B, [b], [1.0])])
        S = oracle.overlap(bas)[:len(cart_list(la)), len(cart_list(la)):]
        E = fk.fock_hermite_e(la, lb, a, A, b, B)
        z = a + b
        K = math.exp(-a * b / z * np.sum((A - B) ** 2)) * (math.pi / z) ** 1.5

        def norm(l, al, c):
            df = lambda n: math.prod(range(n, 0, -2)) if n > 0 else 1.0
            return (2 * al / math.pi) ** 0.75 * (4 * al) ** (l / 2) / math.sqrt(df(2 * c[0] - 1) * df(2 * c[1] - 1) * df(2 * c[2] - 1))

        o = 0
        for i, ca in enumerate(cart_list(la)):
            for j, cb in enumerate(cart_list(lb)):
                n = (ca[0] + cb[0] + 1) * (ca[1] + cb[1] + 1) * (ca[2] + cb[2] + 1)
                val = E[o] * K * norm(la, a, ca) * norm(lb, b, cb)
                assert abs(val - S[i, j]) < 1e-13
                o += n


def _desc(basis):
    return fb._BasisArrays(basis)


def test_build_validation_codes():
    L = fb.lib()
    good = molgen.problem(0).basis

    def build(basis, tau=1e-10):
        arr = _desc(basis)
        out = ctypes.c_void_p()
        rc = L.fock_shellpairs_build(ctypes.byref(arr.desc), None, tau, None, ctypes.byref(out))
        return rc, out

    bad = dict(good)
    bad["l"] = good["l"].copy()
    bad["l"][3] = 4
    assert build(bad)[0] == 2
    bad = dict(good)
    bad["nprim"] = good["nprim"].copy()
    bad["nprim"][0] = 9
    assert build(bad)[0] == 2
    bad = dict(good)
    bad["exps"] = good["exps"].copy()
    bad["exps"][5] = float("nan")
    assert build(bad)[0] == 1
    bad = dict(good)
    bad["exps"] = good["exps"].copy()
    bad["exps"][5] = -1.0
    assert build(bad)[0] == 1
    assert build(good, tau=0.0)[0] == 1
    assert build(good, tau=-1.0)[0] == 1
    out = ctypes.c_void_p()
    assert L.fock_shellpairs_build(None, None, 1e-10, None, ctypes.byref(out)) == 1
    assert L.fock_build_jk(None, None, 1e-10, None, None, None) == 1
    assert L.fock_shellpairs_free(None) == 0
    assert L.fock_nbasis(None) == -1
    assert L.fock_boys_host(13, 1.0, None) == 1
    assert L.fock_hermite_count(4, 0) == -1


def test_opts_layout_and_schedule_validation():
    """The binding's fock_opts matches the library's; schedule entries and
    tune_isolate outside their documented values are rejected before any
    device work."""
    L = fb.lib()
    assert L.fock_opts_size() == ctypes.sizeof(fb.fock_opts)
    assert fb.fock_opts.schedule.offset == 40 and fb.fock_opts.k_mode.offset == 140
    assert fb.fock_opts.k_thresh.offset == 144 and ctypes.sizeof(fb.fock_opts) == 152
    good = molgen.problem(0).basis
    arr = _desc(good)

    def build(o):
        out = ctypes.c_void_p()
        return L.fock_shellpairs_build(ctypes.byref(arr.desc), ctypes.byref(o), 1e-10, None, ctypes.byref(out))

    for v in (3, -2, 64, 5):
        o = fk.make_opts(schedule={(0, 5): v})
        assert build(o) == 1, v
    o = fk.make_opts()
    o.tune_isolate = 2
    assert build(o) == 1
    # exchange mode: only EXACT and DECAY_BOUND, the latter with a positive tau*
    for mode, thr in ((2, 5e-6), (-1, 5e-6), (1, 0.0), (1, -1.0), (1, float("nan"))):
        assert build(fk.make_opts(k_mode=mode, k_thresh=thr)) == 1, (mode, thr)
    o = fk.make_opts(schedule={(5, 2): 8, 12: -1})
    assert fk.schedule_of(o) == {(2, 5): 8, (1, 2): -1}
    assert L.fock_autotune(None, 1, None, None, 1e-10, 3, None, None, None, None) == 1
    D = (ctypes.c_void_p * 1)(1)
    descs = (ctypes.c_void_p * 1)(ctypes.cast(ctypes.pointer(arr.desc), ctypes.c_void_p).value)
    res = fb.fock_opts()
    for reps in (0, 101):
        assert L.fock_autotune(descs, 1, D, None, 1e-10, reps, None, ctypes.byref(res), None, None) == 1
    assert L.fock_autotune(descs, 0, D, None, 1e-10, 3, None, ctypes.byref(res), None, None) == 1


def test_autotune_cache_roundtrip(tmp_path):
    """A stored schedule is found again by workload shape (other geometry,
    same composition) and not for another composition or device."""
    from paper_2407_21445_gb300 import autotune
    p0 = molgen.problem(0)
    bases = [p0.basis]
    cache = str(tmp_path / "tune.json")
    key = autotune.workload_key(bases, 1e-12, None, "GPU-A")
    with open(cache, "w") as f:
        json.dump({key: {"ms_base": 2.0, "ms_tuned": 1.5, "schedule": {"0,5": 8, "2,2": -1}}}, f)
    moved = dict(p0.basis)
    moved["center"] = p0.basis["center"] + 1.0
    o, rec = autotune.tuned_opts([moved], None, 1e-12, cache=cache, device_name="GPU-A")
    assert rec["cached"] and fk.schedule_of(o) == {(0, 5): 8, (2, 2): -1} and o.tune_isolate == 0
    assert autotune.workload_key(bases, 1e-12, None, "GPU-B") != key
    assert autotune.workload_key(bases, 1e-10, None, "GPU-A") != key
    other = molgen.problem(0).basis
    other = dict(other)
    other["nprim"] = other["nprim"].copy()
    other["nprim"][0] = 2
    assert autotune.workload_key([other], 1e-12, None, "GPU-A") != key
