"""CPU FP64 oracle for the J/K build (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package; the GPU library never imports or links it, and
it imports nothing from the GPU package. The C source ``oracle.c`` is compiled
on first use with gcc (or ahead of time by ``build()``).

Every function cites the passage of arXiv:2407.21445 it follows; see the
header of ``oracle.c`` for the readings taken where the paper is garbled.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

SCREEN_NONE, SCREEN_SCHWARZ, SCREEN_DENSITY = 0, 1, 2
# density weighting by the blocks that feed J only (D_ab, D_cd) or K only
# (D_ac, D_ad, D_bc, D_bd): the separate J and K builds (Sec. 4.2, 4.3)
SCREEN_DENSITY_J, SCREEN_DENSITY_K = 3, 4
# primitive pair dropped iff G_[ab] * Gmax < tau * EPS_PRUNE; with the density
# test (SCREEN_DENSITY), primitive quartet skipped iff G_[ab] G_[cd] Dmax < tau * EPS_PRUNE
EPS_PRUNE = 1e-3


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (plain gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            _lib.oracle_boys.argtypes = [i, d, p]
            _lib.oracle_prim_eri.argtypes = [i, i, i, i, d, p, d, p, d, p, d, p, p]
            basis = [i, p, p, p, p, p, p]
            _lib.oracle_norm_coefs.argtypes = basis + [p]
            _lib.oracle_overlap.argtypes = basis + [p]
            _lib.oracle_shell_eri.argtypes = basis + [i, i, i, i, p]
            _lib.oracle_schwarz.argtypes = basis + [p, p]
            _lib.oracle_jk.argtypes = basis + [p, d, i, d, i, i, p, p]
            _lib.oracle_jk_blocks.argtypes = basis + [p, d, i, d, i, p, p, i, p, p]
            _lib.oracle_count.argtypes = basis + [p, d, p]
            _lib.oracle_jk_sample.argtypes = basis + [p, d, i, d, i, i, p, p, p]
            _lib.oracle_kinetic.argtypes = basis + [p]
            _lib.oracle_nuclear.argtypes = basis + [i, p, p, p]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _basis_args(basis: dict):
    arrs = dict(center=np.ascontiguousarray(basis["center"], dtype=np.float64),
                l=np.ascontiguousarray(basis["l"], dtype=np.int32),
                nprim=np.ascontiguousarray(basis["nprim"], dtype=np.int32),
                prim_off=np.ascontiguousarray(basis["prim_off"], dtype=np.int32),
                exps=np.ascontiguousarray(basis["exps"], dtype=np.float64),
                coefs=np.ascontiguousarray(basis["coefs"], dtype=np.float64))
    args = [len(arrs["l"])] + [_ptr(arrs[k]) for k in ("center", "l", "nprim", "prim_off", "exps", "coefs")]
    return args, arrs


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def nbf(basis: dict) -> int:
    return int(sum(ncart(int(l)) for l in basis["l"]))


def boys(mmax: int, T: float) -> np.ndarray:
    """F_m(T), m = 0..mmax (Eq. boys-fn-def)."""
    out = np.zeros(mmax + 1)
    lib().oracle_boys(mmax, float(T), _ptr(out))
    return out


def prim_eri(la, lb, lc, ld, a, A, b, B, c, C, d, D) -> np.ndarray:
    """Primitive [ab|cd] over unnormalised Cartesian Gaussians with unit
    coefficients (Eqs. vrr1, vrr2, hrr); shape [nc(la), nc(lb), nc(lc), nc(ld)]."""
    out = np.zeros(ncart(la) * ncart(lb) * ncart(lc) * ncart(ld))
    vec = [np.ascontiguousarray(x, dtype=np.float64) for x in (A, B, C, D)]
    rc = lib().oracle_prim_eri(la, lb, lc, ld, a, _ptr(vec[0]), b, _ptr(vec[1]), c, _ptr(vec[2]),
                               d, _ptr(vec[3]), _ptr(out))
    if rc:
        raise ValueError("unsupported angular momentum")
    return out.reshape(ncart(la), ncart(lb), ncart(lc), ncart(ld))


def norm_coefs(basis: dict) -> np.ndarray:
    args, keep = _basis_args(basis)
    out = np.zeros_like(keep["exps"])
    lib().oracle_norm_coefs(*args, _ptr(out))
    return out


def overlap(basis: dict) -> np.ndarray:
    """Overlap matrix of the normalised Cartesian basis (Obara-Saika overlap)."""
    args, keep = _basis_args(basis)
    n = nbf(basis)
    S = np.zeros((n, n))
    if lib().oracle_overlap(*args, _ptr(S)):
        raise ValueError("bad basis")
    return S


def kinetic(basis: dict) -> np.ndarray:
    """Kinetic energy matrix, 1/2 sum_x <d_x a|d_x b> (Sec. 2.2 core Hamiltonian)."""
    args, keep = _basis_args(basis)
    n = nbf(basis)
    T = np.zeros((n, n))
    if lib().oracle_kinetic(*args, _ptr(T)):
        raise ValueError("bad basis")
    return T


def nuclear(basis: dict, Z, xyz) -> np.ndarray:
    """Nuclear attraction matrix -sum_C Z_C <a|1/|r-C||b> (Obara-Saika + HRR)."""
    args, keep = _basis_args(basis)
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    n = nbf(basis)
    V = np.zeros((n, n))
    if lib().oracle_nuclear(*args, len(Z), _ptr(Z), _ptr(xyz), _ptr(V)):
        raise ValueError("bad basis")
    return V


def shell_eri(basis: dict, a: int, b: int, c: int, d: int) -> np.ndarray:
    """Contracted (ab|cd) over normalised functions, no screening/pruning."""
    args, keep = _basis_args(basis)
    ls = basis["l"]
    shape = tuple(ncart(int(ls[s])) for s in (a, b, c, d))
    out = np.zeros(int(np.prod(shape)))
    if lib().oracle_shell_eri(*args, a, b, c, d, _ptr(out)):
        raise ValueError("bad basis")
    return out.reshape(shape)


def schwarz(basis: dict):
    """Contracted G_ab [ns, ns] and primitive G_[ab] [ns, ns, 64] (Eqs. cauchy-schwarz 1, 2)."""
    args, keep = _basis_args(basis)
    ns = len(basis["l"])
    G = np.zeros((ns, ns))
    Gp = np.zeros((ns, ns, 64))
    if lib().oracle_schwarz(*args, _ptr(G), _ptr(Gp)):
        raise ValueError("bad basis")
    return G, Gp


def jk(basis: dict, D: np.ndarray, tau: float = 0.0, mode: int = SCREEN_DENSITY,
       eps_prune: float = EPS_PRUNE, symmetric: bool = True, nthreads: int = 0):
    """J_mn = sum (mn|ls) D_ls, K_mn = sum (ml|ns) D_ls (Eq. fock_build) with
    the screening `mode` (0 none, 1 Schwarz, 2 Schwarz x six-block density max,
    3 / 4 Schwarz x the density max of the blocks feeding J / K -- then only J /
    only K is the screened build's) and primitive-pair pruning (eps_prune > 0)."""
    args, keep = _basis_args(basis)
    D = np.ascontiguousarray(D, dtype=np.float64)
    n = nbf(basis)
    assert D.shape == (n, n)
    J = np.zeros((n, n))
    K = np.zeros((n, n))
    rc = lib().oracle_jk(*args, _ptr(D), float(tau), int(mode), float(eps_prune), int(bool(symmetric)),
                         int(nthreads), _ptr(J), _ptr(K))
    if rc:
        raise ValueError("bad basis")
    return J, K


def jk_sample(basis: dict, D: np.ndarray, tau: float, stride: int, nthreads: int = 0,
              mode: int = SCREEN_DENSITY, eps_prune: float = EPS_PRUNE):
    """The symmetric J/K loop over every stride-th outer shell pair only (a
    bounded sample of the full build, used to time the oracle); returns the
    number of Schwarz-passing Cartesian ERIs in the sampled quartets."""
    args, keep = _basis_args(basis)
    D = np.ascontiguousarray(D, dtype=np.float64)
    n = nbf(basis)
    J = np.zeros((n, n))
    K = np.zeros((n, n))
    neri = np.zeros(1)
    rc = lib().oracle_jk_sample(*args, _ptr(D), float(tau), int(mode), float(eps_prune), int(nthreads),
                                int(stride), _ptr(J), _ptr(K), _ptr(neri))
    if rc:
        raise ValueError("bad basis")
    return float(neri[0])


def threads() -> int:
    """Threads the oracle's OpenMP loops use by default."""
    return os.cpu_count() or 1


def jk_blocks(basis: dict, D: np.ndarray, pairs, tau: float, mode: int = SCREEN_DENSITY,
              eps_prune: float = EPS_PRUNE, nthreads: int = 0):
    """Shell-pair blocks (a, b) of J and K computed one by one (no symmetry);
    returns two lists of [nc(a), nc(b)] arrays."""
    args, keep = _basis_args(basis)
    D = np.ascontiguousarray(D, dtype=np.float64)
    pa = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
    pb = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
    ls = basis["l"]
    sizes = [ncart(int(ls[a])) * ncart(int(ls[b])) for a, b in pairs]
    tot = int(sum(sizes))
    Jb = np.zeros(max(tot, 1))
    Kb = np.zeros(max(tot, 1))
    rc = lib().oracle_jk_blocks(*args, _ptr(D), float(tau), int(mode), float(eps_prune), len(pairs),
                                _ptr(pa), _ptr(pb), int(nthreads), _ptr(Jb), _ptr(Kb))
    if rc:
        raise ValueError("bad basis")
    outJ, outK, o = [], [], 0
    for (a, b), s in zip(pairs, sizes):
        shp = (ncart(int(ls[a])), ncart(int(ls[b])))
        outJ.append(Jb[o:o + s].reshape(shp))
        outK.append(Kb[o:o + s].reshape(shp))
        o += s
    return outJ, outK


def count(basis: dict, D: np.ndarray, tau: float) -> dict:
    """Symmetry-unique contracted quartets / Cartesian ERIs passing Schwarz
    (G_ab G_cd >= tau) and the six-block density test."""
    args, keep = _basis_args(basis)
    D = np.ascontiguousarray(D, dtype=np.float64)
    out = np.zeros(4)
    if lib().oracle_count(*args, _ptr(D), float(tau), _ptr(out)):
        raise ValueError("bad basis")
    return dict(quartets_schwarz=int(out[0]), eris_schwarz=int(out[1]),
                quartets_density=int(out[2]), eris_density=int(out[3]))
