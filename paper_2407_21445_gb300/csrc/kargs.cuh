// Kernel argument block shared by the J/K kernels.
#pragma once

#include "fock_impl.h"

namespace fk {

struct KArgs {
  DevPairs dp;
  int nprimtot;
  long long nEtot;
  const double *D;
  const double *Dsh;
  double tau;
  double *J;
  double *K;
  const Unit *units;
  int nunits;
  int *counter;
  int stride;
  const double *boys;
  const ClassTables *tabs;
  // mixed precision: quartets with bound below fp32_cutoff use the FP32 path
  double fp32_cutoff;  // 0 = FP64 only
  const float *Df;     // FP32 copy of D (mixed path)
  const float *boysf;  // FP32 Boys table (same layout)
  const float *Dshf;   // FP32 shell-block maxima (screening pre-test), may be null
  float tau_lo, tau_hi;  // tau (1 -+ 1e-4): FP32 decisions outside this band are exact
  float fp32_cutoff_f;   // fp32_cutoff rounded to FP32
  const MolEntry *mt;  // batched build: per-molecule table (null for one molecule)
  // primitive-quartet screening: [ab|cd] skipped iff G_[ab] G_[cd] Dmax < tau_eps
  double tau_eps;      // tau * prune_eps (0 = off)
  float tau_eps_f;
};

// The molecule a quartet belongs to: its D, J, K, dimension and the block of
// the shell-block maxima, with shell indices made molecule-local.
struct MolView {
  const double *D;
  double *J;
  double *K;
  const float *Df;
  const double *Dsh;
  const float *Dshf;
  int N, s0, ns;
};

__device__ __forceinline__ MolView mol_view(const KArgs &a, int shell) {
  MolView v;
  if (a.mt == nullptr) {
    v.D = a.D;
    v.J = a.J;
    v.K = a.K;
    v.Df = a.Df;
    v.Dsh = a.Dsh;
    v.Dshf = a.Dshf;
    v.N = a.dp.nbf;
    v.s0 = 0;
    v.ns = a.dp.nshell;
  } else {
    const MolEntry &m = a.mt[a.dp.smol[shell]];
    v.D = m.D;
    v.J = m.J;
    v.K = m.K;
    v.Df = m.Df;
    v.Dsh = a.Dsh + m.dsh_off;
    v.Dshf = a.Dshf ? a.Dshf + m.dsh_off : nullptr;
    v.N = m.N;
    v.s0 = m.s0;
    v.ns = m.ns;
  }
  return v;
}

// Density-weighted Schwarz bound G_ab G_cd max|D| over the six blocks
// (Sec. 3.2); returns a negative value when the quartet is screened out.
// The decision is taken on the FP32 units whenever both products are more
// than 1e-4 (relative) away from tau -- FP32 rounding of the inputs and
// products is below 1e-6 -- and in FP64 otherwise, so that it always equals
// the FP64 decision.
__device__ __forceinline__ float quartet_bound(const KArgs &a, const MolView &mv, int sA, int sB, int sC, int sD,
                                               int P, int Q) {
  sA -= mv.s0;
  sB -= mv.s0;
  sC -= mv.s0;
  sD -= mv.s0;
  if (mv.Dshf) {
    const int ns = mv.ns;
    const float *Ds = mv.Dshf;
    const float gf = a.dp.Gf[P] * a.dp.Gf[Q];
    float dm = Ds[sA * ns + sB];
    dm = fmaxf(dm, Ds[sC * ns + sD]);
    dm = fmaxf(dm, Ds[sA * ns + sC]);
    dm = fmaxf(dm, Ds[sA * ns + sD]);
    dm = fmaxf(dm, Ds[sB * ns + sC]);
    dm = fmaxf(dm, Ds[sB * ns + sD]);
    const float bf = gf * dm;
    if (gf < a.tau_lo || bf < a.tau_lo) return -1.0f;
    if (gf > a.tau_hi && bf > a.tau_hi) return bf;
  }
  const double g = a.dp.G[P] * a.dp.G[Q];
  const int ns = mv.ns;
  const double *Ds = mv.Dsh;
  double dm = Ds[sA * ns + sB];
  dm = fmax(dm, Ds[sC * ns + sD]);
  dm = fmax(dm, Ds[sA * ns + sC]);
  dm = fmax(dm, Ds[sA * ns + sD]);
  dm = fmax(dm, Ds[sB * ns + sC]);
  dm = fmax(dm, Ds[sB * ns + sD]);
  const double b = g * dm;
  return (g < a.tau || b < a.tau) ? -1.0f : (float)b;
}

// Primitive-quartet screening inside a contracted quartet that passed
// (Sec. 3.2 primitive Cauchy-Schwarz bound, applied to primitive integrals as
// in the MMD scheme of Sec. 3.3): [ab|cd] is skipped iff
// G_[ab] G_[cd] Dmax < tau * prune_eps, Dmax the six-block maximum of the
// quartet.  The test runs on the FP32 units against a band of 1e-4
// (relative) around the threshold; inside the band it is taken in FP64, so
// that it always equals the FP64 decision.  Each pair's primitives are
// sorted by G_[ab] (descending), so a skip ends the primitive loop.
struct PrimScreen {
  float lo, hi;  // FP32 band on G_[ab] G_[cd]
  float c32;     // mixed precision: primitive quartets of an FP64 quartet with
                 // G_[ab] G_[cd] below this (cutoff / Dmax) run in FP32 (-1 = none)
  int sA, sB, sC, sD;  // molecule-local shells (FP64 Dmax inside the band)
};

__device__ __forceinline__ PrimScreen prim_screen(const KArgs &a, const MolView &mv, int sA, int sB, int sC,
                                                  int sD) {
  PrimScreen ps;
  ps.sA = sA - mv.s0;
  ps.sB = sB - mv.s0;
  ps.sC = sC - mv.s0;
  ps.sD = sD - mv.s0;
  ps.c32 = -1.0f;
  if (a.tau_eps <= 0.0 && a.fp32_cutoff <= 0.0) {
    ps.lo = ps.hi = -1.0f;
    return ps;
  }
  const int ns = mv.ns;
  float dm;
  if (mv.Dshf) {
    const float *Ds = mv.Dshf;
    dm = Ds[ps.sA * ns + ps.sB];
    dm = fmaxf(dm, Ds[ps.sC * ns + ps.sD]);
    dm = fmaxf(dm, Ds[ps.sA * ns + ps.sC]);
    dm = fmaxf(dm, Ds[ps.sA * ns + ps.sD]);
    dm = fmaxf(dm, Ds[ps.sB * ns + ps.sC]);
    dm = fmaxf(dm, Ds[ps.sB * ns + ps.sD]);
  } else {
    const double *Ds = mv.Dsh;
    double d = Ds[ps.sA * ns + ps.sB];
    d = fmax(d, Ds[ps.sC * ns + ps.sD]);
    d = fmax(d, Ds[ps.sA * ns + ps.sC]);
    d = fmax(d, Ds[ps.sA * ns + ps.sD]);
    d = fmax(d, Ds[ps.sB * ns + ps.sC]);
    d = fmax(d, Ds[ps.sB * ns + ps.sD]);
    dm = (float)d;
  }
  if (a.fp32_cutoff > 0.0) ps.c32 = a.fp32_cutoff_f / dm;
  if (a.tau_eps <= 0.0) {
    ps.lo = ps.hi = -1.0f;
    return ps;
  }
  const float t = a.tau_eps_f / dm;
  ps.lo = t * (1.0f - 1e-4f);
  ps.hi = t * (1.0f + 1e-4f);
  return ps;
}

// Mixed precision at primitive granularity: inside a quartet whose bound is
// at least the FP32 cutoff, primitive quartet [ab|cd] is evaluated in FP32
// when its own bound G_[ab] G_[cd] Dmax is below the cutoff.  Both sides of
// the split use this one FP32 expression; with each pair's primitives sorted
// by G_[ab] it is non-increasing along either primitive loop.
__device__ __forceinline__ bool prim_fp32(const KArgs &a, const PrimScreen &ps, int ip, int jq) {
  return a.dp.Gpf[ip] * a.dp.Gpf[jq] < ps.c32;
}

// true = skip primitive quartet (ip | jq)
__device__ __forceinline__ bool prim_skip(const KArgs &a, const MolView &mv, const PrimScreen &ps, int ip, int jq) {
  const float x = a.dp.Gpf[ip] * a.dp.Gpf[jq];
  if (x < ps.lo) return true;
  if (x > ps.hi || ps.lo < 0.0f) return false;
  const int ns = mv.ns;
  const double *Ds = mv.Dsh;
  double d = Ds[ps.sA * ns + ps.sB];
  d = fmax(d, Ds[ps.sC * ns + ps.sD]);
  d = fmax(d, Ds[ps.sA * ns + ps.sC]);
  d = fmax(d, Ds[ps.sA * ns + ps.sD]);
  d = fmax(d, Ds[ps.sB * ns + ps.sC]);
  d = fmax(d, Ds[ps.sB * ns + ps.sD]);
  return a.dp.Gp[ip] * a.dp.Gp[jq] * d < a.tau_eps;
}

// Density-weighted Schwarz test of quartet (P|Q) (Sec. 3.2): true = skip.
__device__ __forceinline__ bool screened(const KArgs &a, const MolView &mv, int sA, int sB, int sC, int sD, int P,
                                         int Q) {
  return quartet_bound(a, mv, sA, sB, sC, sD, P, Q) < 0.0f;
}

// Next work unit for the calling warp (lane 0 draws from the tier counter).
__device__ __forceinline__ int next_unit(int *counter, int lane) {
  int u = 0;
  if (lane == 0) u = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, u, 0);
}

}  // namespace fk
