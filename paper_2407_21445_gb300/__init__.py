"""GB300-native Coulomb/exchange (J/K) builder (arXiv:2407.21445 hot path).

The compute path is the in-tree CUDA library libfock.so (C ABI in
include/fock.h); this package holds its build script and a ctypes binding.

Usage (device tensors are torch float64 CUDA tensors; the basis is a dict of
numpy arrays: center [nshell*3] bohr, l, nprim, prim_off, exps, coefs and
optionally atom, as produced by molgen.make_basis):

    import torch, paper_2407_21445_gb300 as fk
    b = fk.JKBuilder(basis, 1e-10)                        # shell pairs, Schwarz factors, work lists
    J, K = b.build(torch.tensor(D, device="cuda"))        # one J/K build on the current stream

    opts = fk.make_opts(precision=fk.FOCK_MIXED, fp32_cutoff=1e-5)
    bm = fk.JKBuilder(basis, 1e-10, opts)                 # FP32 below the density-weighted bound

    hs = [fk.fock_shellpairs_build(bs, 1e-10) for bs in bases]
    fk.fock_build_jk_batched(hs, Ds, 1e-10, Js, Ks)       # many molecules, one graph replay

    from paper_2407_21445_gb300 import autotune
    opts, rec = autotune.tuned_opts([basis], [Dt], 1e-10, cache="tune.json")  # measured schedule

The SCF driver (scf.RHF, scf.sad_guess) and the learned initial density
(guess.LearnedGuess.load(".../guess_mlp.npz")) build on the same library.
"""
from .fock import (FOCK_FP64, FOCK_MIXED, MLP, NCLASS, FockError, JKBuilder, fock_autotune, fock_boys_host,
                   fock_boys_table_info, fock_build_jk, fock_build_jk_batched, fock_hermite_count, fock_hermite_e, fock_kernels_per_build, fock_nbasis, fock_one_electron,
                   fock_shellpairs_build, fock_shellpairs_free, fock_status_string, fock_stream_status,
                   fock_work_stats, lib, make_opts, schedule_of)

__all__ = ["FOCK_FP64", "FOCK_MIXED", "MLP", "NCLASS", "FockError", "JKBuilder", "fock_autotune", "fock_boys_host", "fock_boys_table_info",
           "fock_build_jk", "fock_build_jk_batched", "fock_hermite_count", "fock_hermite_e", "fock_kernels_per_build", "fock_nbasis", "fock_one_electron",
           "fock_shellpairs_build", "fock_shellpairs_free", "fock_status_string", "fock_stream_status",
           "fock_work_stats", "lib", "make_opts", "schedule_of"]
