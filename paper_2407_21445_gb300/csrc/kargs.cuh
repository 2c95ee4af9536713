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
};

// Density-weighted Schwarz bound G_ab G_cd max|D| over the six blocks
// (Sec. 3.2); returns a negative value when the quartet is screened out.
__device__ __forceinline__ double quartet_bound(const KArgs &a, int sA, int sB, int sC, int sD, int P, int Q) {
  const double g = a.dp.G[P] * a.dp.G[Q];
  const int ns = a.dp.nshell;
  const double *Ds = a.Dsh;
  double dm = Ds[sA * ns + sB];
  dm = fmax(dm, Ds[sC * ns + sD]);
  dm = fmax(dm, Ds[sA * ns + sC]);
  dm = fmax(dm, Ds[sA * ns + sD]);
  dm = fmax(dm, Ds[sB * ns + sC]);
  dm = fmax(dm, Ds[sB * ns + sD]);
  const double b = g * dm;
  return (g < a.tau || b < a.tau) ? -1.0 : b;
}

// Density-weighted Schwarz test of quartet (P|Q) (Sec. 3.2): true = skip.
__device__ __forceinline__ bool screened(const KArgs &a, int sA, int sB, int sC, int sD, int P, int Q) {
  const double g = a.dp.G[P] * a.dp.G[Q];
  const int ns = a.dp.nshell;
  const double *Ds = a.Dsh;
  double dm = Ds[sA * ns + sB];
  dm = fmax(dm, Ds[sC * ns + sD]);
  dm = fmax(dm, Ds[sA * ns + sC]);
  dm = fmax(dm, Ds[sA * ns + sD]);
  dm = fmax(dm, Ds[sB * ns + sC]);
  dm = fmax(dm, Ds[sB * ns + sD]);
  return g < a.tau || g * dm < a.tau;
}

// Next work unit for the calling warp (lane 0 draws from the tier counter).
__device__ __forceinline__ int next_unit(int *counter, int lane) {
  int u = 0;
  if (lane == 0) u = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, u, 0);
}

}  // namespace fk
