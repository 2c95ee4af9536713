// fock_build_jk_noalloc: the J/K build with its per-call scratch in a fixed
// device array owned by the library instead of memory obtained per call.
//
// Who needs this: callers that must not allocate device memory while they
// run, such as services that reserve their whole memory budget at start-up,
// applications whose allocator policy forbids the CUDA runtime's
// stream-ordered pool (cudaMallocAsync), and real-time loops where an
// allocation could stall.  fock_build_jk takes its scratch from the pool on
// every call; this variant takes it from g_noalloc_scratch below and calls no
// allocation routine at all.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "fock_impl.h"

namespace fk {
namespace {

// Per-call scratch of fock_build_jk_noalloc: the shell-block density maxima
// (nshell^2 doubles) followed by one work counter per tier.  Every GPU that
// loads the library keeps this array for the life of the process.
constexpr size_t kNoallocBytes = 4u << 20;  // 4 MiB: up to 724 shells
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch per device.  In host code the symbol
// name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with the device current.
void *s_scratch_addr[64];
std::mutex s_scratch_mu;

cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(s_scratch_mu);
  if (!s_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    s_scratch_addr[dev] = p;
  }
  *out = s_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace fk

using namespace fk;

extern "C" fock_status fock_build_jk_noalloc(const fock_shellpairs *sp, const double *D, double schwarz_thresh,
                                             double *J, double *K, cudaStream_t stream) {
  if (!sp || !D || !J || !K) return FOCK_ERR_INVALID_ARG;
  if (!(schwarz_thresh >= sp->tau_build) || !isfinite(schwarz_thresh)) return FOCK_ERR_INVALID_ARG;
  const int ns = sp->nshell, n = sp->nbf;
  const size_t nt = sp->tiers.size();
  const size_t dsh_bytes = sizeof(double) * (size_t)ns * ns;
  const size_t cnt_off = (dsh_bytes + 255) & ~(size_t)255;
  const size_t need = cnt_off + sizeof(int) * (nt + 1);
  if (need > kNoallocBytes) return FOCK_ERR_INVALID_ARG;  // basis too large for the fixed array
  void *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return FOCK_ERR_CUDA;
  char *scratch = (char *)base;
  double *Dsh = (double *)scratch;  // fully rewritten by the density preparation kernel
  int *counters = (int *)(scratch + cnt_off);
  // The counters keep the previous call's values: they must start at zero.
  e = cudaMemsetAsync(counters, 0, sizeof(int) * (nt + 1), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(J, 0, sizeof(double) * (size_t)n * n, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(K, 0, sizeof(double) * (size_t)n * n, stream);
  if (e == cudaSuccess) e = launch_dprep(D, n, sp->dev.sbf, sp->dev.sl, ns, Dsh, stream);
  for (size_t t = 0; t < nt && e == cudaSuccess; ++t)
    e = launch_jk_tier(sp->tiers[t], sp->dev, D, Dsh, schwarz_thresh, sp->prune_eps, J, K, counters + t, nullptr,
                       stream);
  if (e == cudaSuccess) e = launch_symmetrize(J, K, n, stream);
  if (e == cudaSuccess) return FOCK_OK;
  return e == cudaErrorMemoryAllocation ? FOCK_ERR_OOM : FOCK_ERR_CUDA;
}
