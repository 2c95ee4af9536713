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

// Per-call scratch of fock_build_jk_noalloc, laid out as in fock_build_jk
// (scratch_layout): the shell-block density maxima (nshell^2 doubles), two
// work counters per tier and one spare, the FP32 copy of D (N^2 floats, mixed
// precision only), the FP32 shell-block maxima (nshell^2 floats) and, in the
// decay-bound exchange mode, the bounds (nshell^2 floats), distance bins and
// fit, each part 256-byte aligned.  Every GPU that loads the library keeps
// this array for the life of the process.
constexpr size_t kNoallocBytes = 4u << 20;  // 4 MiB: FP64 handles up to 591 shells
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

}  // namespace
}  // namespace fk

using namespace fk;

extern "C" fock_status fock_build_jk_noalloc(const fock_shellpairs *sp, const double *D, double schwarz_thresh,
                                             double *J, double *K, cudaStream_t stream) {
  if (!sp || !D || (!J && !K)) return FOCK_ERR_INVALID_ARG;
  if (!(schwarz_thresh >= sp->tau_build) || !isfinite(schwarz_thresh)) return FOCK_ERR_INVALID_ARG;
  const int ns = sp->nshell, n = sp->nbf;
  const size_t nt = sp->tiers.size();
  const bool mixed = sp->opts.precision == FOCK_MIXED && sp->opts.fp32_cutoff > 0.0;
  const ScratchLayout L = scratch_layout(sp);  // the layout fock_build_jk uses
  if (L.total > kNoallocBytes) return FOCK_ERR_INVALID_ARG;  // basis too large for the fixed array
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
  int *counters = (int *)(scratch + L.cnt_off);
  float *Df = mixed ? (float *)(scratch + L.df_off) : nullptr;  // rewritten by k_dprep
  float *Dshf = (float *)(scratch + L.dshf_off);                // rewritten by k_dprep
  CallParts cp;
  cp.parts = (J ? 1 : 0) | (K ? 2 : 0);
  const bool decay = sp->opts.k_mode == FOCK_K_DECAY_BOUND && K;
  const bool chk = sync_each_launch();
  const char *where = "memset";
  // The counters keep the previous call's values: they must start at zero
  // (the decay-bound bins are cleared by their own launch).
  e = cudaMemsetAsync(counters, 0, sizeof(int) * (2 * nt + 1), stream);
  if (e == cudaSuccess && J) e = cudaMemsetAsync(J, 0, sizeof(double) * (size_t)n * n, stream);
  if (e == cudaSuccess && K) e = cudaMemsetAsync(K, 0, sizeof(double) * (size_t)n * n, stream);
  if (e == cudaSuccess) {
    where = "k_dprep";
    e = launch_dprep(D, n, sp->dev.sbf, sp->dev.sl, ns, Dsh, stream, Df, Dshf);
    if (e == cudaSuccess && chk) e = cudaStreamSynchronize(stream);
  }
  if (e == cudaSuccess && decay) {
    where = "decay bound";
    float *W = (float *)(scratch + L.w_off);
    e = launch_decay_bound(sp->dev, Dsh, sp->decay_nbins, (double *)(scratch + L.bins_off),
                           (double *)(scratch + L.hl_off), W, stream, sp->dev.Gn, Dshf,
                           (float *)(scratch + L.t_off), (float *)(scratch + L.gdg_off), sp->opts.k_thresh);
    if (e == cudaSuccess && chk) e = cudaStreamSynchronize(stream);
    cp.Wsh = W;
    cp.k_thresh = sp->opts.k_thresh;
  }
  char tier_name[64];
  for (size_t t = 0; t < nt && e == cudaSuccess; ++t) {
    snprintf(tier_name, sizeof(tier_name), "k_jk tier %zu (G=%d, smem=%zu)", t, sp->tiers[t].G, sp->tiers[t].smem);
    where = tier_name;
    e = launch_jk_tier(sp->tiers[t], sp->dev, D, Dsh, schwarz_thresh, sp->prune_eps, J, K, counters + t,
                       counters + nt + t, stream, Df, sp->opts.fp32_cutoff, Dshf, cp);
    if (e == cudaSuccess && chk) e = cudaStreamSynchronize(stream);
  }
  if (e == cudaSuccess) {
    where = "k_symmetrize";
    e = launch_symmetrize(J, K, n, stream);
    if (e == cudaSuccess && chk) e = cudaStreamSynchronize(stream);
  }
  return cuda_status(e, where);
}
