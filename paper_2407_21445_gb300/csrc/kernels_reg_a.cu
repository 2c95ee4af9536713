// Register-kernel instantiations with an (s s| bra: (ss|ss) .. (ss|fs).
#include "kernels_reg.cuh"
#include "reg_dispatch.h"

namespace fk {

#define FK_REG_LIST(X) \
  X(0, 0, 0, 0, 0, 0)  \
  X(0, 1, 0, 0, 1, 0)  \
  X(0, 2, 0, 0, 1, 1)  \
  X(0, 3, 0, 0, 2, 0)  \
  X(0, 4, 0, 0, 2, 1)  \
  X(0, 6, 0, 0, 3, 0)
#include "reg_dispatch.inc"

cudaError_t launch_reg_a(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st) {
  return reg_launch_impl(cb, ck, a, blocks, threads, st);
}
cudaError_t occupancy_reg_a(int cb, int ck, int threads, bool mixed, int *per_sm) {
  return reg_occupancy_impl(cb, ck, threads, mixed, per_sm);
}

}  // namespace fk
