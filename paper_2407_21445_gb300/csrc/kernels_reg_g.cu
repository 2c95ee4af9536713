// FP32-only register kernels (k_reg32) of the d-shell class pairs with total L = 5
// and of (dd|pp).
#include "kernels_reg.cuh"
#include "reg_dispatch.h"

namespace fk {

#define FK_REG32_LIST(X) \
  X(5, 1, 2, 2, 1, 0) \
  X(1, 5, 1, 0, 2, 2) \
  X(4, 2, 2, 1, 1, 1) \
  X(2, 4, 1, 1, 2, 1) \
  X(4, 3, 2, 1, 2, 0) \
  X(3, 4, 2, 0, 2, 1) \
  X(5, 2, 2, 2, 1, 1)

bool reg32_listed_g(int cb, int ck) {
#define FK_R32_HAS(CB, CK, LA, LB, LC, LD) \
  if (cb == CB && ck == CK) return true;
  FK_REG32_LIST(FK_R32_HAS)
#undef FK_R32_HAS
  return false;
}

cudaError_t launch_reg32_g(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st) {
#define FK_R32_LAUNCH(CB, CK, LA, LB, LC, LD)                                                           \
  if (cb == CB && ck == CK) {                                                                            \
    const int sm = reg32_smem_bytes<LA, LB, LC, LD>(threads);                                           \
    if (sm > 48 * 1024) {                                                                                \
      cudaError_t e = cudaFuncSetAttribute(k_reg32<LA, LB, LC, LD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm); \
      if (e != cudaSuccess) return e;                                                                    \
    }                                                                                                    \
    k_reg32<LA, LB, LC, LD><<<blocks, threads, sm, st>>>(a);                                             \
    return cudaGetLastError();                                                                           \
  }
  FK_REG32_LIST(FK_R32_LAUNCH)
#undef FK_R32_LAUNCH
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_reg32_g(int cb, int ck, int threads, int *per_sm) {
#define FK_R32_OCC(CB, CK, LA, LB, LC, LD)                                                              \
  if (cb == CB && ck == CK) {                                                                            \
    const int sm = reg32_smem_bytes<LA, LB, LC, LD>(threads);                                           \
    if (sm > 48 * 1024) {                                                                                \
      cudaError_t e = cudaFuncSetAttribute(k_reg32<LA, LB, LC, LD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm); \
      if (e != cudaSuccess) return e;                                                                    \
    }                                                                                                    \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_reg32<LA, LB, LC, LD>, threads, sm);    \
  }
  FK_REG32_LIST(FK_R32_OCC)
#undef FK_R32_OCC
  return cudaErrorInvalidValue;
}

}  // namespace fk
