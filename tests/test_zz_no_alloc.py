"""fock_build_jk_noalloc: the allocation-free variant of fock_build_jk, for
callers that cannot allocate device memory while they run (fixed memory
budgets, allocator policies without the stream-ordered pool, real-time
loops).  Called through the C ABI, it must reproduce fock_build_jk on
consecutive calls (its fixed scratch array keeps the previous call's
contents), in FP64 and in mixed precision, and refuse bases too large for
that array.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import molgen

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-7}  # FP64 and mixed-precision tolerances of the parity tests


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    import paper_2407_21445_gb300 as fk
    L = fk.lib()
    L.fock_build_jk_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
    L.fock_build_jk_noalloc.restype = ctypes.c_int32
    return torch, fk, L


def _noalloc(L, torch, handle, D, tau, J, K):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(None if t is None else t.data_ptr())  # noqa: E731
    return L.fock_build_jk_noalloc(handle, ctypes.c_void_p(D.data_ptr()), tau, ptr(J), ptr(K), stream)


@pytest.mark.parametrize("config,precision", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_noalloc_matches_fock_build_jk_twice(env, config, precision):
    torch, fk, L = env
    p = molgen.problem(config)
    b = fk.JKBuilder(p.basis, p.tau, fk.make_opts(precision=precision))
    D = torch.tensor(p.D, device="cuda", dtype=torch.float64)
    Jr, Kr = b.build(D)
    torch.cuda.synchronize()
    Jr, Kr = Jr.cpu().numpy(), Kr.cpu().numpy()
    for call in range(2):
        J = torch.full_like(D, float("nan"))
        K = torch.full_like(D, float("nan"))
        assert _noalloc(L, torch, b.handle, D, p.tau, J, K) == 0
        torch.cuda.synchronize()
        assert fk.fock_stream_status() == 0
        ej = float(np.abs(J.cpu().numpy() - Jr).max())
        ek = float(np.abs(K.cpu().numpy() - Kr).max())
        assert ej <= TOL[precision] and ek <= TOL[precision], (call, ej, ek)
    b.close()


def test_noalloc_decay_mode_k_only_twice(env):
    """The decay-bound exchange mode with only K requested (the fixed array
    then also holds the bounds, the distance bins and the GDG products)."""
    torch, fk, L = env
    p = molgen.problem(1, carbons=12)
    b = fk.JKBuilder(p.basis, p.tau, fk.make_opts(k_mode=1, k_thresh=5e-6))
    D = torch.tensor(p.D, device="cuda", dtype=torch.float64)
    _, Kr = b.build(D, parts="k")
    torch.cuda.synchronize()
    for call in range(2):
        K = torch.full_like(D, float("nan"))
        assert _noalloc(L, torch, b.handle, D, p.tau, None, K) == 0
        torch.cuda.synchronize()
        assert fk.fock_stream_status() == 0
        assert float((K - Kr).abs().max()) <= TOL[0], call
    b.close()


def _s_shell_basis(n, seed=11):
    rng = np.random.Generator(np.random.PCG64(seed))
    return molgen.single_shell_basis([(0, rng.uniform(-40, 40, 3), [0.5], [1.0]) for _ in range(n)])


def test_noalloc_size_limit(env):
    """The fixed array holds 12 nshell^2 bytes plus the counters for FP64
    handles up to 591 shells; 592 shells are refused without any work."""
    torch, fk, L = env
    for n, ok in ((591, True), (592, False)):
        b = fk.JKBuilder(_s_shell_basis(n), 1e-8)
        D = torch.eye(n, device="cuda", dtype=torch.float64) * 0.5
        J = torch.zeros_like(D)
        K = torch.zeros_like(D)
        rc = _noalloc(L, torch, b.handle, D, 1e-8, J, K)
        torch.cuda.synchronize()
        if ok:
            assert rc == 0 and fk.fock_stream_status() == 0
            Jr, Kr = b.build(D)
            torch.cuda.synchronize()
            assert float((J - Jr).abs().max()) <= TOL[0] and float((K - Kr).abs().max()) <= TOL[0]
        else:
            assert rc == 1  # FOCK_ERR_INVALID_ARG
            assert float(J.abs().max()) == 0.0 and float(K.abs().max()) == 0.0
        b.close()


def test_noalloc_rejects_basis_beyond_array(env):
    torch, fk, L = env
    # 800 s shells (800^2 doubles of shell-block maxima exceed the 4 MiB array)
    rng = np.random.Generator(np.random.PCG64(11))
    shells = [(0, rng.uniform(-40, 40, 3), [0.5], [1.0]) for _ in range(800)]
    bas = molgen.single_shell_basis(shells)
    b = fk.JKBuilder(bas, 1e-8)
    D = torch.eye(800, device="cuda", dtype=torch.float64)
    J = torch.zeros_like(D)
    K = torch.zeros_like(D)
    assert _noalloc(L, torch, b.handle, D, 1e-8, J, K) == 1  # FOCK_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert float(J.abs().max()) == 0.0
