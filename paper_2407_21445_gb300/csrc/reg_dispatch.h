// Launch/occupancy entry points of the per-class register kernels.
#pragma once

#include "kargs.cuh"

namespace fk {
cudaError_t launch_reg_a(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg_a(int cb, int ck, int threads, int *per_sm);
cudaError_t launch_reg_b(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg_b(int cb, int ck, int threads, int *per_sm);
cudaError_t launch_reg_c(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg_c(int cb, int ck, int threads, int *per_sm);
cudaError_t launch_reg_d(int cb, int ck, const KArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t occupancy_reg_d(int cb, int ck, int threads, int *per_sm);
}  // namespace fk
