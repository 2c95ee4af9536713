// Register-kernel instantiations with total L = 4 (s-s bra or ket with d-d or f-p).
#include "kernels_reg.cuh"
#include "reg_dispatch.h"

namespace fk {

#define FK_REG_LIST(X) \
  X(0, 5, 0, 0, 2, 2) \
  X(5, 0, 2, 2, 0, 0) \
  X(0, 7, 0, 0, 3, 1) \
  X(7, 0, 3, 1, 0, 0)
#include "reg_dispatch.inc"

cudaError_t launch_reg_c(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st) {
  return reg_launch_impl(cb, ck, a, blocks, threads, st);
}
cudaError_t occupancy_reg_c(int cb, int ck, int threads, bool mixed, int *per_sm) {
  return reg_occupancy_impl(cb, ck, threads, mixed, per_sm);
}

}  // namespace fk
