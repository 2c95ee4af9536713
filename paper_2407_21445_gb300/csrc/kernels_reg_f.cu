// Register-kernel instantiations with total L = 4 (d-s bra).
#include "kernels_reg.cuh"
#include "reg_dispatch.h"

namespace fk {

#define FK_REG_LIST(X) \
  X(3, 2, 2, 0, 1, 1) \
  X(3, 3, 2, 0, 2, 0)
#include "reg_dispatch.inc"

cudaError_t launch_reg_f(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st) {
  return reg_launch_impl(cb, ck, a, blocks, threads, st);
}
cudaError_t occupancy_reg_f(int cb, int ck, int threads, bool mixed, int *per_sm) {
  return reg_occupancy_impl(cb, ck, threads, mixed, per_sm);
}

}  // namespace fk
