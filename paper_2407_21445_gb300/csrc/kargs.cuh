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
  // which matrices are built: 1 = J, 2 = K, 3 = both (fused)
  int parts;
  // decay-bound exchange mode (Sec. 4.3.1): per shell pair (x, y) the bound
  // H exp(-Lambda (|XY| - R_x - R_y)) of the density block a K_xy
  // contribution is contracted with (+inf where the exponent is not
  // positive); null in the exact mode
  const float *Wsh;
  float k_thresh_f;    // tau*
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
  const float *Wsh;
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
    v.Wsh = a.Wsh;
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
    v.Wsh = nullptr;  // the batched build runs the exact exchange test only
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
static __device__ __noinline__ float quartet_bound_parts(const KArgs &a, const MolView &mv, int sA, int sB, int sC,
                                                        int sD, int P, int Q);

// FULL = false: the fused J+K build with the exact test only (kernels compiled
// without the J-only / K-only / decay-bound code, which costs registers).
template <bool FULL = true>
__device__ __forceinline__ float quartet_bound(const KArgs &a, const MolView &mv, int sA, int sB, int sC, int sD,
                                               int P, int Q) {
  if constexpr (FULL) {
    if (a.parts != 3 || mv.Wsh) return quartet_bound_parts(a, mv, sA, sB, sC, sD, P, Q);
  }
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

// FP32 pre-test against tau with an exact FP64 decision inside the band
// (1 = at least tau, 0 = below)
__device__ __forceinline__ bool at_least_tau(const KArgs &a, float xf, double gx, const double *Ds, int i0, int i1,
                                             int i2, int i3, int nblk) {
  if (xf < a.tau_lo) return false;
  if (xf > a.tau_hi) return true;
  double d = Ds[i0];
  d = fmax(d, Ds[i1]);
  if (nblk > 2) d = fmax(fmax(d, Ds[i2]), Ds[i3]);
  return gx * d >= a.tau;
}

// Quartet test of a build of J only, K only, or of the decay-bound exchange
// mode: the Coulomb part weighs G_ab G_cd with max(|D_ab|, |D_cd|), the
// exchange part with max(|D_ac|, |D_ad|, |D_bc|, |D_bd|) (exact mode, against
// tau) or with the decay bound max(W_ac, W_ad, W_bc, W_bd) (against tau*,
// Sec. 4.3.1); a quartet is evaluated when a part that is built needs it.
// Returns the exact-density bound of the built parts (the mixed-precision
// decision) or a negative value when the quartet is skipped.
static __device__ __noinline__ float quartet_bound_parts(const KArgs &a, const MolView &mv, int sA, int sB, int sC,
                                                        int sD, int P, int Q) {
  sA -= mv.s0;
  sB -= mv.s0;
  sC -= mv.s0;
  sD -= mv.s0;
  const int ns = mv.ns;
  const int iab = sA * ns + sB, icd = sC * ns + sD, iac = sA * ns + sC, iad = sA * ns + sD, ibc = sB * ns + sC,
            ibd = sB * ns + sD;
  const float gf = a.dp.Gf[P] * a.dp.Gf[Q];
  const double g = a.dp.G[P] * a.dp.G[Q];
  // Schwarz test itself (Sec. 3.2)
  if (gf < a.tau_lo || (!(gf > a.tau_hi) && g < a.tau)) return -1.0f;
  const float *Dsf = mv.Dshf;
  float dj = 0.0f, dk = 0.0f;
  bool keep = false;
  if (a.parts & 1) {
    dj = Dsf ? fmaxf(Dsf[iab], Dsf[icd]) : (float)fmax(mv.Dsh[iab], mv.Dsh[icd]);
    keep = at_least_tau(a, gf * dj, g, mv.Dsh, iab, icd, 0, 0, 2);
  }
  if (a.parts & 2) {
    dk = Dsf ? fmaxf(fmaxf(Dsf[iac], Dsf[iad]), fmaxf(Dsf[ibc], Dsf[ibd]))
             : (float)fmax(fmax(mv.Dsh[iac], mv.Dsh[iad]), fmax(mv.Dsh[ibc], mv.Dsh[ibd]));
    if (!keep) {
      if (mv.Wsh) {
        const float *W = mv.Wsh;
        const float w = fmaxf(fmaxf(W[iac], W[iad]), fmaxf(W[ibc], W[ibd]));
        keep = gf * w >= a.k_thresh_f;
      } else {
        keep = at_least_tau(a, gf * dk, g, mv.Dsh, iac, iad, ibc, ibd, 4);
      }
    }
  }
  return keep ? gf * fmaxf(dj, dk) : -1.0f;
}

// Primitive-quartet screening inside a contracted quartet that passed
// (Sec. 3.2 primitive Cauchy-Schwarz bound, applied to primitive integrals as
// in the MMD scheme of Sec. 3.3): [ab|cd] is skipped iff
// G_[ab] G_[cd] Dmax < tau * prune_eps, Dmax the six-block maximum of the
// quartet.  The test runs on the FP32 units against a band of 1e-4
// (relative) around the threshold; inside the band it is taken in FP64, so
// that it always equals the FP64 decision.  Each pair's primitives are
// sorted by G_[ab] (descending), so a skip ends the primitive loop.
// Density maximum over the shell blocks the built parts are contracted with
// (parts 3: all six; J: ab, cd; K: ac, ad, bc, bd); molecule-local shells.
template <class T>
__device__ __forceinline__ T dmax_parts(int parts, const T *Ds, int ns, int sA, int sB, int sC, int sD) {
  T d = T(0);
  if (parts & 1) d = fmax(Ds[sA * ns + sB], Ds[sC * ns + sD]);
  if (parts & 2) {
    d = fmax(d, fmax(Ds[sA * ns + sC], Ds[sA * ns + sD]));
    d = fmax(d, fmax(Ds[sB * ns + sC], Ds[sB * ns + sD]));
  }
  return d;
}

struct PrimScreen {
  float lo, hi;  // FP32 band on G_[ab] G_[cd]
  float c32;     // mixed precision: primitive quartets of an FP64 quartet with
                 // G_[ab] G_[cd] below this (cutoff / Dmax) run in FP32 (-1 = none)
  int sA, sB, sC, sD;  // molecule-local shells (FP64 Dmax inside the band)
  int parts;           // the density blocks weighed (as KArgs::parts)
};

template <bool FULL = true>
__device__ __forceinline__ PrimScreen prim_screen(const KArgs &a, const MolView &mv, int sA, int sB, int sC,
                                                  int sD) {
  const int parts = FULL ? a.parts : 3;
  PrimScreen ps;
  ps.parts = parts;
  ps.sA = sA - mv.s0;
  ps.sB = sB - mv.s0;
  ps.sC = sC - mv.s0;
  ps.sD = sD - mv.s0;
  ps.c32 = -1.0f;
  if (a.tau_eps <= 0.0 && a.fp32_cutoff <= 0.0) {
    ps.lo = ps.hi = -1.0f;
    return ps;
  }
  float dm;
  if (mv.Dshf)
    dm = dmax_parts<float>(parts, mv.Dshf, mv.ns, ps.sA, ps.sB, ps.sC, ps.sD);
  else
    dm = (float)dmax_parts<double>(parts, mv.Dsh, mv.ns, ps.sA, ps.sB, ps.sC, ps.sD);
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
  const double d = dmax_parts<double>(ps.parts, mv.Dsh, mv.ns, ps.sA, ps.sB, ps.sC, ps.sD);
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
