// Launch/occupancy entry points of the per-class register kernels.
#pragma once

#include "kargs.cuh"

namespace fk {
cudaError_t launch_reg_a(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg_a(int cb, int ck, int threads, bool mixed, int *per_sm);
cudaError_t launch_reg_b(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg_b(int cb, int ck, int threads, bool mixed, int *per_sm);
cudaError_t launch_reg_c(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg_c(int cb, int ck, int threads, bool mixed, int *per_sm);
cudaError_t launch_reg_d(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg_d(int cb, int ck, int threads, bool mixed, int *per_sm);
cudaError_t launch_reg_e(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg_e(int cb, int ck, int threads, bool mixed, int *per_sm);
cudaError_t launch_reg_f(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg_f(int cb, int ck, int threads, bool mixed, int *per_sm);

cudaError_t launch_reg32_g(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg32_g(int cb, int ck, int threads, int *per_sm);
cudaError_t launch_reg32_h(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg32_h(int cb, int ck, int threads, int *per_sm);

bool reg32_listed_g(int cb, int ck);
bool reg32_listed_h(int cb, int ck);
// Class pairs (bra class, ket class) with an FP32-only register kernel
// (k_reg32), as instantiated: total angular momentum 5 (l <= 3) and (dd|pp)
// (the other total-6 pairs would spill kilobytes per thread).
inline bool reg32_available(int cb, int ck) { return reg32_listed_g(cb, ck) || reg32_listed_h(cb, ck); }
inline cudaError_t launch_reg32(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st) {
  cudaError_t e = launch_reg32_g(cb, ck, a, blocks, threads, st);
  if (e == cudaErrorInvalidValue) e = launch_reg32_h(cb, ck, a, blocks, threads, st);
  return e;
}
inline cudaError_t occupancy_reg32(int cb, int ck, int threads, int *per_sm) {
  cudaError_t e = occupancy_reg32_g(cb, ck, threads, per_sm);
  if (e == cudaErrorInvalidValue) e = occupancy_reg32_h(cb, ck, threads, per_sm);
  return e;
}

// Launch / occupancy of the register kernel of class pair (cb, ck), whichever
// translation unit instantiates it (cudaErrorInvalidValue if none does).
inline cudaError_t launch_reg(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st) {
  cudaError_t (*const fns[])(int, int, const KArgs &, int, int, cudaStream_t) = {
      launch_reg_a, launch_reg_b, launch_reg_c, launch_reg_d, launch_reg_e, launch_reg_f};
  cudaError_t e = cudaErrorInvalidValue;
  for (auto fn : fns) {
    e = fn(cb, ck, a, blocks, threads, st);
    if (e != cudaErrorInvalidValue) break;
  }
  return e;
}
inline cudaError_t occupancy_reg(int cb, int ck, int threads, bool mixed, int *per_sm) {
  cudaError_t (*const fns[])(int, int, int, bool, int *) = {occupancy_reg_a, occupancy_reg_b, occupancy_reg_c,
                                                           occupancy_reg_d, occupancy_reg_e, occupancy_reg_f};
  cudaError_t e = cudaErrorInvalidValue;
  for (auto fn : fns) {
    e = fn(cb, ck, threads, mixed, per_sm);
    if (e != cudaErrorInvalidValue) break;
  }
  return e;
}
}  // namespace fk
