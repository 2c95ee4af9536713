"""Thin ctypes binding of libfock.so (include/fock.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; PyTorch supplies device
memory and streams. Functions keep the C names. There is no CPU fallback: a
missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import _build

FOCK_OK = 0
FOCK_FP64, FOCK_MIXED = 0, 1
STATUS_NAMES = ["FOCK_OK", "FOCK_ERR_INVALID_ARG", "FOCK_ERR_UNSUPPORTED_L", "FOCK_ERR_NONFINITE",
                "FOCK_ERR_OOM", "FOCK_ERR_CUDA", "FOCK_ERR_TIMEOUT", "FOCK_ERR_NOT_CONVERGED"]


class FockError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}")


class fock_basis_desc(ctypes.Structure):
    _fields_ = [("nshell", ctypes.c_int32), ("center", ctypes.c_void_p), ("l", ctypes.c_void_p),
                ("nprim", ctypes.c_void_p), ("prim_off", ctypes.c_void_p), ("exps", ctypes.c_void_p),
                ("coefs", ctypes.c_void_p), ("atom", ctypes.c_void_p)]


NCLASS = 10  # shell-pair classes ss .. ff


class fock_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("fp32_cutoff", ctypes.c_double), ("prune_eps", ctypes.c_double),
                ("group_override", ctypes.c_int32), ("warp_scratch", ctypes.c_int32), ("reg_max_L", ctypes.c_int32),
                ("tune_isolate", ctypes.c_int32), ("schedule", ctypes.c_int8 * (NCLASS * NCLASS)),
                ("k_mode", ctypes.c_int32), ("k_thresh", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libfock.so, building it in-tree first if it is absent or stale."""
    global _lib
    with _lock:
        if _lib is None:
            checked = os.environ.get("FOCK_CHECKED_LIB") == "1"  # bounds-checked diagnostic build
            path = _build.build(checked=checked)
            if not os.path.exists(path):
                raise RuntimeError(f"libfock.so missing at {path}")
            L = ctypes.CDLL(path)
            p, d, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int32
            L.fock_shellpairs_build.argtypes = [ctypes.POINTER(fock_basis_desc), ctypes.POINTER(fock_opts), d, p,
                                                ctypes.POINTER(p)]
            L.fock_shellpairs_build.restype = i
            L.fock_shellpairs_free.argtypes = [p]
            L.fock_shellpairs_free.restype = i
            L.fock_nbasis.argtypes = [p]
            L.fock_nbasis.restype = i
            L.fock_kernels_per_build.argtypes = [p]
            L.fock_kernels_per_build.restype = i
            L.fock_build_jk.argtypes = [p, p, d, p, p, p]
            L.fock_build_jk.restype = i
            L.fock_build_jk_batched.argtypes = [p, i, p, d, p, p, p]
            L.fock_build_jk_batched.restype = i
            L.fock_work_stats.argtypes = [p, p, d, p]
            L.fock_work_stats.restype = i
            L.fock_stream_status.argtypes = [p]
            L.fock_stream_status.restype = i
            L.fock_one_electron.argtypes = [ctypes.POINTER(fock_basis_desc), i, p, p, p, p, p, p]
            L.fock_one_electron.restype = i
            L.fock_mlp_create.argtypes = [i, i, i, i, ctypes.c_uint64, ctypes.POINTER(p)]
            L.fock_mlp_create.restype = i
            L.fock_mlp_free.argtypes = [p]
            L.fock_mlp_free.restype = i
            L.fock_mlp_num_params.argtypes = [p]
            L.fock_mlp_num_params.restype = ctypes.c_int64
            L.fock_mlp_get_params.argtypes = [p, p, p]
            L.fock_mlp_get_params.restype = i
            L.fock_mlp_set_params.argtypes = [p, p]
            L.fock_mlp_set_params.restype = i
            L.fock_mlp_forward.argtypes = [p, p, i, p, p]
            L.fock_mlp_forward.restype = i
            L.fock_mlp_loss_backward.argtypes = [p, p, p, p, i, d, p, p]
            L.fock_mlp_loss_backward.restype = i
            L.fock_mlp_step.argtypes = [p, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, p]
            L.fock_mlp_step.restype = i
            L.fock_mlp_zero_grad.argtypes = [p, p]
            L.fock_mlp_zero_grad.restype = i
            L.fock_debug_bounds.argtypes = [p]
            L.fock_debug_bounds.restype = i
            L.fock_last_error.argtypes = []
            L.fock_last_error.restype = ctypes.c_char_p
            L.fock_status_string.argtypes = [i]
            L.fock_status_string.restype = ctypes.c_char_p
            L.fock_boys_table_info.argtypes = [p]
            L.fock_boys_table_info.restype = i
            L.fock_boys_host.argtypes = [i, d, p]
            L.fock_boys_host.restype = i
            L.fock_hermite_count.argtypes = [i, i]
            L.fock_hermite_count.restype = i
            L.fock_hermite_e.argtypes = [i, i, d, p, d, p, p]
            L.fock_hermite_e.restype = i
            L.fock_decay_bound.argtypes = [p, p, p, p, p, p]
            L.fock_decay_bound.restype = i
            L.fock_build_jk_noalloc.argtypes = [p, p, d, p, p, p]
            L.fock_build_jk_noalloc.restype = i
            L.fock_opts_size.argtypes = []
            L.fock_opts_size.restype = i
            L.fock_autotune.argtypes = [p, i, p, ctypes.POINTER(fock_opts), d, i, p, ctypes.POINTER(fock_opts), p,
                                        p]
            L.fock_autotune.restype = i
            if L.fock_opts_size() != ctypes.sizeof(fock_opts):
                raise RuntimeError("fock_opts layout differs between include/fock.h and the binding")
            _lib = L
    return _lib


def declared_symbols():
    """Names of the entry points declared in include/fock.h."""
    with open(os.path.join(_build.INCLUDE, "fock.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"FOCK_API\s+[\w\s\*]+?\b(fock_\w+)\s*\(", text)))


def _check(rc: int, where: str):
    if rc != FOCK_OK:
        detail = lib().fock_last_error().decode() if rc == 5 else ""
        raise FockError(rc, f"{where} [{detail}]" if detail else where)


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _tensor_ptr(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class _BasisArrays:
    def __init__(self, basis: dict):
        self.center = np.ascontiguousarray(basis["center"], dtype=np.float64)
        self.l = np.ascontiguousarray(basis["l"], dtype=np.int32)
        self.nprim = np.ascontiguousarray(basis["nprim"], dtype=np.int32)
        self.prim_off = np.ascontiguousarray(basis["prim_off"], dtype=np.int32)
        self.exps = np.ascontiguousarray(basis["exps"], dtype=np.float64)
        self.coefs = np.ascontiguousarray(basis["coefs"], dtype=np.float64)
        atom = basis.get("atom")
        self.atom = None if atom is None else np.ascontiguousarray(atom, dtype=np.int32)
        self.desc = fock_basis_desc(len(self.l), _np_ptr(self.center), _np_ptr(self.l), _np_ptr(self.nprim),
                                    _np_ptr(self.prim_off), _np_ptr(self.exps), _np_ptr(self.coefs),
                                    None if self.atom is None else _np_ptr(self.atom))


def make_opts(precision=FOCK_FP64, fp32_cutoff=1e-5, prune_eps=1e-3, group_override=0, warp_scratch=0,
              reg_max_L=0, schedule=None, k_mode=0, k_thresh=5e-6) -> fock_opts:
    o = fock_opts()
    o.k_mode = k_mode
    o.k_thresh = k_thresh
    o.reg_max_L = reg_max_L
    o.warp_scratch = warp_scratch
    o.precision = precision
    o.fp32_cutoff = fp32_cutoff
    o.prune_eps = prune_eps
    o.group_override = group_override
    if schedule is not None:
        for k, v in dict(schedule).items():
            c1, c2 = sorted(k) if isinstance(k, tuple) else divmod(int(k), NCLASS)
            o.schedule[c1 * NCLASS + c2] = int(v)
    return o


def schedule_of(o: fock_opts) -> dict:
    """Non-default schedule entries {(c1, c2): value} of an options struct."""
    return {(i // NCLASS, i % NCLASS): int(v) for i, v in enumerate(o.schedule) if v != 0}


def fock_shellpairs_build(basis: dict, schwarz_thresh: float, opts: fock_opts | None = None, stream=None):
    """Returns an opaque handle (ctypes.c_void_p); see include/fock.h."""
    arr = _BasisArrays(basis)
    out = ctypes.c_void_p()
    rc = lib().fock_shellpairs_build(ctypes.byref(arr.desc), ctypes.byref(opts) if opts is not None else None,
                                     float(schwarz_thresh), _stream_handle(stream), ctypes.byref(out))
    _check(rc, "fock_shellpairs_build")
    return out


def fock_shellpairs_free(handle):
    _check(lib().fock_shellpairs_free(handle), "fock_shellpairs_free")


def fock_nbasis(handle) -> int:
    return int(lib().fock_nbasis(handle))


def fock_kernels_per_build(handle) -> int:
    return int(lib().fock_kernels_per_build(handle))


def _opt_tensor_ptr(t, name):
    return None if t is None else _tensor_ptr(t, name)


def fock_build_jk(handle, D, schwarz_thresh: float, J, K, stream=None):
    """J and K of D; one of J, K may be None (only the other is built)."""
    rc = lib().fock_build_jk(handle, _tensor_ptr(D, "D"), float(schwarz_thresh), _opt_tensor_ptr(J, "J"),
                             _opt_tensor_ptr(K, "K"), _stream_handle(stream))
    _check(rc, "fock_build_jk")


def fock_decay_bound(handle, D, nshell: int, stream=None):
    """(H, Lambda, R[nshell], G[nshell]) of the density decay bound (Sec. 4.3.1)."""
    ns = int(nshell)
    hl = np.zeros(2)
    R = np.zeros(ns)
    G = np.zeros(ns)
    rc = lib().fock_decay_bound(handle, _tensor_ptr(D, "D"), _np_ptr(hl), _np_ptr(R), _np_ptr(G),
                                _stream_handle(stream))
    _check(rc, "fock_decay_bound")
    return float(hl[0]), float(hl[1]), R, G


def fock_build_jk_noalloc(handle, D, schwarz_thresh: float, J, K, stream=None):
    rc = lib().fock_build_jk_noalloc(handle, _tensor_ptr(D, "D"), float(schwarz_thresh), _opt_tensor_ptr(J, "J"),
                                     _opt_tensor_ptr(K, "K"), _stream_handle(stream))
    _check(rc, "fock_build_jk_noalloc")


def fock_opts_size() -> int:
    return int(lib().fock_opts_size())


def fock_build_jk_batched(handles, Ds, schwarz_thresh: float, Js, Ks, stream=None):
    n = len(handles)
    H = (ctypes.c_void_p * n)(*[h.value for h in handles])
    Dp = (ctypes.c_void_p * n)(*[_tensor_ptr(x, "D").value for x in Ds])
    Jp = (ctypes.c_void_p * n)(*[_tensor_ptr(x, "J").value for x in Js])
    Kp = (ctypes.c_void_p * n)(*[_tensor_ptr(x, "K").value for x in Ks])
    rc = lib().fock_build_jk_batched(H, n, Dp, float(schwarz_thresh), Jp, Kp, _stream_handle(stream))
    _check(rc, "fock_build_jk_batched")


def fock_autotune(bases, Ds, schwarz_thresh: float, opts: fock_opts | None = None, reps: int = 3, stream=None):
    """Measured per-class-pair schedule for the workload (bases, device
    densities Ds); returns (tuned fock_opts, [ms with base, ms tuned],
    {(c1, c2): ms of that class pair with the base schedule})."""
    n = len(bases)
    arrs = [_BasisArrays(b) for b in bases]
    descs = (ctypes.c_void_p * n)(*[ctypes.cast(ctypes.pointer(a.desc), ctypes.c_void_p).value for a in arrs])
    Dp = (ctypes.c_void_p * n)(*[_tensor_ptr(x, "D").value for x in Ds])
    out = fock_opts()
    ms = np.zeros(2)
    pair = np.zeros(NCLASS * NCLASS)
    rc = lib().fock_autotune(descs, n, Dp, ctypes.byref(opts) if opts is not None else None, float(schwarz_thresh),
                             int(reps), _stream_handle(stream), ctypes.byref(out), _np_ptr(ms), _np_ptr(pair))
    _check(rc, "fock_autotune")
    return out, [float(ms[0]), float(ms[1])], {(i // NCLASS, i % NCLASS): float(v) for i, v in enumerate(pair) if v > 0}


def fock_work_stats(handle, D_host: np.ndarray, schwarz_thresh: float) -> dict:
    D_host = np.ascontiguousarray(D_host, dtype=np.float64)
    out = np.zeros(10)
    _check(lib().fock_work_stats(handle, _np_ptr(D_host), float(schwarz_thresh), _np_ptr(out)), "fock_work_stats")
    keys = ["quartets_schwarz", "eris_schwarz", "quartets_evaluated", "eris_evaluated", "prim_quartets",
            "flops_model", "prim_pairs", "pairs", "quartets_fp32", "flops_model_fp32"]
    return {k: float(v) for k, v in zip(keys, out)}


def fock_stream_status(stream=None) -> int:
    return int(lib().fock_stream_status(_stream_handle(stream)))


def fock_one_electron(basis: dict, Z, xyz, stream=None):
    """Overlap, kinetic and nuclear-attraction matrices (device float64 tensors)."""
    import torch
    arr = _BasisArrays(basis)
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    n = int(sum((int(l) + 1) * (int(l) + 2) // 2 for l in arr.l))
    S, T, V = (torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(3))
    rc = lib().fock_one_electron(ctypes.byref(arr.desc), len(Z), _np_ptr(Z), _np_ptr(xyz), _tensor_ptr(S, "S"),
                                 _tensor_ptr(T, "T"), _tensor_ptr(V, "V"), _stream_handle(stream))
    _check(rc, "fock_one_electron")
    return S, T, V


def fock_debug_bounds():
    out = np.zeros(2, dtype=np.int64)
    _check(lib().fock_debug_bounds(_np_ptr(out)), "fock_debug_bounds")
    return int(out[0]), int(out[1])


def fock_last_error() -> str:
    return lib().fock_last_error().decode()


def fock_status_string(st: int) -> str:
    return lib().fock_status_string(int(st)).decode()


def fock_boys_table_info() -> dict:
    out = np.zeros(4)
    _check(lib().fock_boys_table_info(_np_ptr(out)), "fock_boys_table_info")
    return dict(h=out[0], ngrid=int(out[1]), norders=int(out[2]), tmax=out[3])


def fock_boys_host(mmax: int, T: float) -> np.ndarray:
    F = np.zeros(mmax + 1)
    _check(lib().fock_boys_host(int(mmax), float(T), _np_ptr(F)), "fock_boys_host")
    return F


def fock_hermite_count(la: int, lb: int) -> int:
    return int(lib().fock_hermite_count(int(la), int(lb)))


def fock_hermite_e(la: int, lb: int, alpha: float, A, beta: float, B) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    out = np.zeros(max(fock_hermite_count(la, lb), 1))
    _check(lib().fock_hermite_e(int(la), int(lb), float(alpha), _np_ptr(A), float(beta), _np_ptr(B), _np_ptr(out)),
           "fock_hermite_e")
    return out


def _f32_ptr(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


# --- atom-pair MLP (fock_mlp_*), one wrapper per entry point ---------------

def fock_mlp_create(nin: int, nhidden: int, nout: int, max_batch: int, seed: int = 0):
    h = ctypes.c_void_p()
    _check(lib().fock_mlp_create(nin, nhidden, nout, max_batch, seed, ctypes.byref(h)), "fock_mlp_create")
    return h


def fock_mlp_free(handle):
    _check(lib().fock_mlp_free(handle), "fock_mlp_free")


def fock_mlp_num_params(handle) -> int:
    return int(lib().fock_mlp_num_params(handle))


def fock_mlp_get_params(handle, params: np.ndarray | None, grads: np.ndarray | None):
    """Copies the FP32 master parameters and/or gradients into the given host arrays."""
    _check(lib().fock_mlp_get_params(handle, None if params is None else _np_ptr(params),
                                     None if grads is None else _np_ptr(grads)), "fock_mlp_get_params")


def fock_mlp_set_params(handle, params: np.ndarray):
    _check(lib().fock_mlp_set_params(handle, _np_ptr(params)), "fock_mlp_set_params")


def fock_mlp_forward(handle, X, n: int, Y, stream=None):
    _check(lib().fock_mlp_forward(handle, _f32_ptr(X, "X"), n, _f32_ptr(Y, "Y"), _stream_handle(stream)),
           "fock_mlp_forward")


def fock_mlp_loss_backward(handle, X, T, mask, n: int, norm: float, stream=None) -> float:
    out = np.zeros(1, dtype=np.float32)
    _check(lib().fock_mlp_loss_backward(handle, _f32_ptr(X, "X"), _f32_ptr(T, "T"),
                                        None if mask is None else _f32_ptr(mask, "mask"), n, float(norm),
                                        _np_ptr(out), _stream_handle(stream)), "fock_mlp_loss_backward")
    return float(out[0])


def fock_mlp_step(handle, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
    _check(lib().fock_mlp_step(handle, lr, beta1, beta2, eps, weight_decay, _stream_handle(stream)), "fock_mlp_step")


def fock_mlp_zero_grad(handle, stream=None):
    _check(lib().fock_mlp_zero_grad(handle, _stream_handle(stream)), "fock_mlp_zero_grad")


class MLP:
    """The library's atom-pair MLP (fock_mlp_*): BF16 weights, FP32 accumulation."""

    def __init__(self, nin: int, nhidden: int, nout: int, max_batch: int, seed: int = 0):
        self.nin, self.nhidden, self.nout, self.max_batch = nin, nhidden, nout, max_batch
        self.handle = fock_mlp_create(nin, nhidden, nout, max_batch, seed)
        self.nparam = fock_mlp_num_params(self.handle)

    def params(self):
        p = np.zeros(self.nparam, dtype=np.float32)
        fock_mlp_get_params(self.handle, p, None)
        return p

    def grads(self):
        g = np.zeros(self.nparam, dtype=np.float32)
        fock_mlp_get_params(self.handle, None, g)
        return g

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparam
        fock_mlp_set_params(self.handle, p)

    def forward(self, X, Y=None, stream=None):
        import torch
        if Y is None:
            Y = torch.empty((X.shape[0], self.nout), dtype=torch.float32, device=X.device)
        fock_mlp_forward(self.handle, X, X.shape[0], Y, stream)
        return Y

    def loss_backward(self, X, T, mask=None, norm=None, stream=None) -> float:
        norm = float(mask.sum()) if (norm is None and mask is not None) else float(norm or T.numel())
        return fock_mlp_loss_backward(self.handle, X, T, mask, X.shape[0], norm, stream)

    def step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
        fock_mlp_step(self.handle, lr, beta1, beta2, eps, weight_decay, stream)

    def zero_grad(self, stream=None):
        fock_mlp_zero_grad(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            fock_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class JKBuilder:
    """Owns a shell-pair handle; builds J and K for device densities."""

    def __init__(self, basis: dict, schwarz_thresh: float, opts: fock_opts | None = None, stream=None):
        self.tau = float(schwarz_thresh)
        self.handle = fock_shellpairs_build(basis, schwarz_thresh, opts, stream)
        self.nbf = fock_nbasis(self.handle)
        self.nshell = len(basis["l"])

    def build(self, D, J=None, K=None, tau=None, stream=None, parts="jk"):
        """J and K of D (parts "jk"), or only J ("j") or only K ("k"), the other
        returned as None."""
        import torch
        if J is None and "j" in parts:
            J = torch.empty_like(D)
        if K is None and "k" in parts:
            K = torch.empty_like(D)
        fock_build_jk(self.handle, D, self.tau if tau is None else tau, J if "j" in parts else None,
                      K if "k" in parts else None, stream)
        return (J if "j" in parts else None), (K if "k" in parts else None)

    def decay_bound(self, D, stream=None):
        return fock_decay_bound(self.handle, D, self.nshell, stream)

    def stats(self, D_host, tau=None) -> dict:
        return fock_work_stats(self.handle, D_host, self.tau if tau is None else tau)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            fock_shellpairs_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
