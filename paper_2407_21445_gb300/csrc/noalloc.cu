// fock_build_jk_noalloc: the J/K build with its per-call scratch in a fixed
// device array owned by the library instead of memory obtained per call.
//
// Who needs this: callers that must not allocate device memory while they
// run, such as services that reserve their whole memory budget at start-up,
// applications whose allocator policy forbids the CUDA runtime's
// stream-ordered pool (cudaMallocAsync), and real-time loops where an
// allocation could stall.  fock_build_jk takes its scratch from the pool on
// every call; this variant takes it from g_noalloc_scratch below and calls no
// allocation routine at all.  It launches the same kernels with the same
// arguments as fock_build_jk, in both precisions.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "fock_impl.h"

namespace fk {
namespace {

// Per-call scratch of fock_build_jk_noalloc, laid out as in fock_build_jk:
// the shell-block density maxima (nshell^2 doubles), two work counters per
// tier and one spare, the FP32 copy of D (N^2 floats, mixed precision only)
// and the FP32 shell-block maxima (nshell^2 floats), each part 256-byte
// aligned.  Every GPU that loads the library keeps this array for the life of
// the process.
constexpr size_t kNoallocBytes = 4u << 20;  // 4 MiB: FP64 handles up to 591 shells
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace fk

using namespace fk;

extern "C" fock_status fock_build_jk_noalloc(const fock_shellpairs *sp, const double *D, double schwarz_thresh,
                                             double *J, double *K, cudaStream_t stream) {
  if (!sp || !D || !J || !K) return FOCK_ERR_INVALID_ARG;
  if (!(schwarz_thresh >= sp->tau_build) || !isfinite(schwarz_thresh)) return FOCK_ERR_INVALID_ARG;
  const int ns = sp->nshell, n = sp->nbf;
  const size_t nt = sp->tiers.size();
  const bool mixed = sp->opts.precision == FOCK_MIXED && sp->opts.fp32_cutoff > 0.0;
  const size_t cnt_off = align256(sizeof(double) * (size_t)ns * ns);
  const size_t df_off = align256(cnt_off + sizeof(int) * (2 * nt + 1));
  const size_t dshf_off = mixed ? align256(df_off + sizeof(float) * (size_t)n * n) : df_off;
  const size_t need = dshf_off + sizeof(float) * (size_t)ns * ns;
  if (need > kNoallocBytes) return FOCK_ERR_INVALID_ARG;  // basis too large for the fixed array
  // In host code g_noalloc_scratch names a host-side stand-in; the device
  // address comes from cudaGetSymbolAddress with the device current.  It is
  // looked up on every call: the array belongs to the library's module in
  // the device's current context, and a context torn down and created again
  // (cudaDeviceReset) may place it elsewhere.  The lookup is cheap once the
  // module is loaded; the first call on a device loads it.
  void *base = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress");
  char *scratch = (char *)base;
  double *Dsh = (double *)scratch;  // fully rewritten by the density preparation kernel
  int *counters = (int *)(scratch + cnt_off);
  float *Df = mixed ? (float *)(scratch + df_off) : nullptr;  // rewritten by k_dprep
  float *Dshf = (float *)(scratch + dshf_off);                // rewritten by k_dprep
  const bool chk = sync_each_launch();
  const char *where = "memset";
  // The counters keep the previous call's values: they must start at zero.
  e = cudaMemsetAsync(counters, 0, sizeof(int) * (2 * nt + 1), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(J, 0, sizeof(double) * (size_t)n * n, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(K, 0, sizeof(double) * (size_t)n * n, stream);
  if (e == cudaSuccess) {
    where = "k_dprep";
    e = launch_dprep(D, n, sp->dev.sbf, sp->dev.sl, ns, Dsh, stream, Df, Dshf);
    if (e == cudaSuccess && chk) e = cudaStreamSynchronize(stream);
  }
  char tier_name[64];
  for (size_t t = 0; t < nt && e == cudaSuccess; ++t) {
    snprintf(tier_name, sizeof(tier_name), "k_jk tier %zu (G=%d, smem=%zu)", t, sp->tiers[t].G, sp->tiers[t].smem);
    where = tier_name;
    e = launch_jk_tier(sp->tiers[t], sp->dev, D, Dsh, schwarz_thresh, sp->prune_eps, J, K, counters + t,
                       counters + nt + t, stream, Df, sp->opts.fp32_cutoff, Dshf);
    if (e == cudaSuccess && chk) e = cudaStreamSynchronize(stream);
  }
  if (e == cudaSuccess) {
    where = "k_symmetrize";
    e = launch_symmetrize(J, K, n, stream);
    if (e == cudaSuccess && chk) e = cudaStreamSynchronize(stream);
  }
  return cuda_status(e, where);
}
