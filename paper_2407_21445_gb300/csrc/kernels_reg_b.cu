// Register-kernel instantiations with a p, d or f bra pair, total L <= 3.
#include "kernels_reg.cuh"
#include "reg_dispatch.h"

namespace fk {

#define FK_REG_LIST(X) \
  X(1, 0, 1, 0, 0, 0)  \
  X(1, 1, 1, 0, 1, 0)  \
  X(1, 2, 1, 0, 1, 1)  \
  X(1, 3, 1, 0, 2, 0)  \
  X(2, 0, 1, 1, 0, 0)  \
  X(2, 1, 1, 1, 1, 0)  \
  X(3, 0, 2, 0, 0, 0)  \
  X(3, 1, 2, 0, 1, 0)  \
  X(4, 0, 2, 1, 0, 0)  \
  X(6, 0, 3, 0, 0, 0)
#include "reg_dispatch.inc"

cudaError_t launch_reg_b(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st) {
  return reg_launch_impl(cb, ck, a, blocks, threads, st);
}
cudaError_t occupancy_reg_b(int cb, int ck, int threads, bool mixed, int *per_sm) {
  return reg_occupancy_impl(cb, ck, threads, mixed, per_sm);
}

}  // namespace fk
