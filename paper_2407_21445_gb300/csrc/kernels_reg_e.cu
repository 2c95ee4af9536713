// Register-kernel instantiations with total L = 4 (p-s with d-p or f-s).
#include "kernels_reg.cuh"
#include "reg_dispatch.h"

namespace fk {

#define FK_REG_LIST(X) \
  X(1, 4, 1, 0, 2, 1) \
  X(4, 1, 2, 1, 1, 0) \
  X(1, 6, 1, 0, 3, 0) \
  X(6, 1, 3, 0, 1, 0)
#include "reg_dispatch.inc"

cudaError_t launch_reg_e(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st) {
  return reg_launch_impl(cb, ck, a, blocks, threads, st);
}
cudaError_t occupancy_reg_e(int cb, int ck, int threads, bool mixed, int *per_sm) {
  return reg_occupancy_impl(cb, ck, threads, mixed, per_sm);
}

}  // namespace fk
