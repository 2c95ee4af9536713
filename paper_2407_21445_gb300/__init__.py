"""GB300-native Coulomb/exchange (J/K) builder (arXiv:2407.21445 hot path).

The compute path is the in-tree CUDA library libfock.so (C ABI in
include/fock.h); this package holds its build script and a ctypes binding.
"""
from .fock import (FOCK_FP64, FOCK_MIXED, MLP, NCLASS, FockError, JKBuilder, fock_autotune, fock_boys_host,
                   fock_boys_table_info, fock_build_jk, fock_build_jk_batched, fock_hermite_count, fock_hermite_e, fock_kernels_per_build, fock_nbasis, fock_one_electron,
                   fock_shellpairs_build, fock_shellpairs_free, fock_status_string, fock_stream_status,
                   fock_work_stats, lib, make_opts, schedule_of)

__all__ = ["FOCK_FP64", "FOCK_MIXED", "MLP", "NCLASS", "FockError", "JKBuilder", "fock_autotune", "fock_boys_host", "fock_boys_table_info",
           "fock_build_jk", "fock_build_jk_batched", "fock_hermite_count", "fock_hermite_e", "fock_kernels_per_build", "fock_nbasis", "fock_one_electron",
           "fock_shellpairs_build", "fock_shellpairs_free", "fock_status_string", "fock_stream_status",
           "fock_work_stats", "lib", "make_opts", "schedule_of"]
