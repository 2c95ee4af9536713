// Per-class register kernels: one thread owns one contracted shell quartet
// of a fixed angular-momentum class (la lb|lc ld) with total L <= 4 (k_reg;
// FP32 quartets of total L = 5 and (dd|pp) in k_reg32); every loop has a
// compile-time trip count and the intermediates (Boys seeds, Hermite
// integrals R, half-transformed Y) are registers, the contracted ERIs too
// except in the largest classes, which keep them in per-thread shared memory.
// Same McMurchie-Davidson steps and digestion as the group kernel in
// kernels_jk.cu (Sec. 4.1 Eqs. MD def, EabP def1-3; Sec. 3.2 digestion).
#pragma once

#include <type_traits>
#include <utility>

#include "device_common.cuh"
#include "kargs.cuh"

namespace fk {

struct TUV {
  int t, u, v;
};

__host__ __device__ constexpr int ct_hidx(int t, int u, int v) {
  return (t + u + v) * (t + u + v + 1) * (t + u + v + 2) / 6 + (u + v) * (u + v + 1) / 2 + v;
}

// inverse of ct_hidx
__host__ __device__ constexpr TUV ct_hvec(int e) {
  int d = 0;
  while (nherm(d) <= e) ++d;
  int r = e - (d > 0 ? nherm(d - 1) : 0);
  int k = 0;
  while (r > k) {
    r -= k + 1;
    ++k;
  }
  return TUV{d - k, k - r, r};
}

// Cartesian component i of a shell of angular momentum l (x^l first).
__host__ __device__ constexpr TUV ct_cart(int l, int i) {
  int k = 0;
  while (i > k) {
    i -= k + 1;
    ++k;
  }
  return TUV{l - k, k - i, i};
}

__host__ __device__ constexpr int ct_box(int la, int ia, int lb, int ib) {
  return (ct_cart(la, ia).t + ct_cart(lb, ib).t + 1) * (ct_cart(la, ia).u + ct_cart(lb, ib).u + 1) *
         (ct_cart(la, ia).v + ct_cart(lb, ib).v + 1);
}

// offset of Cartesian pair k = ia*ncart(lb)+ib in a primitive pair's E block
__host__ __device__ constexpr int ct_eoff(int la, int lb, int k) {
  int o = 0;
  for (int j = 0; j < k; ++j) o += ct_box(la, j / ncart(lb), lb, j % ncart(lb));
  return o;
}

// Compile-time loop: f(std::integral_constant<int, i>) for i = 0..N-1, so
// that every index derived from i is a constant expression.
template <class F, int... Is>
__device__ __forceinline__ void sfor_impl(F &&f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void sfor(F &&f) {
  sfor_impl(f, std::make_integer_sequence<int, N>{});
}
#define FK_CI(x) decltype(x)::value

// R^{(0)}_{tuv}, t+u+v <= L, from the seeds F[n] = pref (-2 alpha)^n F_n(T)
// by R^{(n)}_{t,u,v} = (t-1) R^{(n+1)}_{t-2,u,v} + X_PQ R^{(n+1)}_{t-1,u,v}
// (or the same along y, z for t = 0).
template <int L, class Real>
__device__ __forceinline__ void hermite_r_reg(const Real (&F)[L + 1], Real X, Real Y, Real Z, Real (&R)[nherm(L)]) {
  Real W[L + 1][nherm(L)];
  W[L][0] = F[L];
  sfor<L>([&](auto li) {
    constexpr int n = L - 1 - FK_CI(li);
    W[n][0] = F[n];
    sfor<nherm(L - n) - 1>([&](auto ei) {
      constexpr int e = FK_CI(ei) + 1;
      constexpr TUV h = ct_hvec(e);
      if constexpr (h.t > 0) {
        Real v = X * W[n + 1][ct_hidx(h.t - 1, h.u, h.v)];
        if constexpr (h.t > 1) v = fma((Real)(h.t - 1), W[n + 1][ct_hidx(h.t - 2, h.u, h.v)], v);
        W[n][e] = v;
      } else if constexpr (h.u > 0) {
        Real v = Y * W[n + 1][ct_hidx(h.t, h.u - 1, h.v)];
        if constexpr (h.u > 1) v = fma((Real)(h.u - 1), W[n + 1][ct_hidx(h.t, h.u - 2, h.v)], v);
        W[n][e] = v;
      } else {
        Real v = Z * W[n + 1][ct_hidx(h.t, h.u, h.v - 1)];
        if constexpr (h.v > 1) v = fma((Real)(h.v - 1), W[n + 1][ct_hidx(h.t, h.u, h.v - 2)], v);
        W[n][e] = v;
      }
    });
  });
  sfor<nherm(L)>([&](auto ei) { R[FK_CI(ei)] = W[0][FK_CI(ei)]; });
}

// Classes whose contracted-ERI accumulator and half-transformed Y together
// would overflow the register file keep the accumulator in shared memory
// (one column per thread, [element][thread] layout, no bank conflicts).
template <int LA, int LB, int LC, int LD>
__host__ __device__ constexpr bool reg_eri_in_smem() {
  return ncart(LA) * ncart(LB) * ncart(LC) * ncart(LD) + nherm(LA + LB) * ncart(LC) * ncart(LD) > 140;
}
template <int LA, int LB, int LC, int LD>
__host__ __device__ constexpr int reg_smem_bytes(int threads) {
  return reg_eri_in_smem<LA, LB, LC, LD>() ? ncart(LA) * ncart(LB) * ncart(LC) * ncart(LD) * threads * 8 : 0;
}

// FP32 primitive quartet [ab|cd] (pair-relative centres, FP32 Boys table and
// Hermite recursion) added into the half-transformed Y[p][cd].
template <int LA, int LB, int LC, int LD>
__device__ __forceinline__ void prim_f32_ket(const KArgs &a, const float4 &PA, int jq, float ACx, float ACy,
                                             float ACz, float (&Y)[nherm(LA + LB) * ncart(LC) * ncart(LD)]) {
  constexpr int ND = ncart(LD), NCD = ncart(LC) * ND;
  constexpr int NHAB = nherm(LA + LB), L = LA + LB + LC + LD, NHL = nherm(L);
  const DevPairs &dp = a.dp;
  const float4 QC = dp.paf[jq];
  const float X = PA.x - QC.x + ACx, Yd = PA.y - QC.y + ACy, Z = PA.z - QC.z + ACz;
  const float rs = rsqrtf(PA.w + QC.w);
  const float alpha = (PA.w * QC.w) * (rs * rs);
  const float T = alpha * fmaf(X, X, fmaf(Yd, Yd, Z * Z));
  float F[L + 1];
  boys_seeds_f32<L>(a.boysf, T, rs, -2.0f * alpha, F);
  float R[NHL];
  hermite_r_reg<L, float>(F, X, Yd, Z, R);
  const float *__restrict__ EQ = dp.Ef + dp.eoff[jq];
  sfor<NCD>([&](auto kci) {
    constexpr int kc = FK_CI(kci);
    constexpr TUV c = ct_cart(LC, kc / ND), d = ct_cart(LD, kc % ND);
    constexpr int TY = c.u + d.u + 1, TZ = c.v + d.v + 1, NQ = (c.t + d.t + 1) * TY * TZ;
    constexpr int e0 = ct_eoff(LC, LD, kc);
    sfor<NQ>([&](auto qi) {
      constexpr int qq = FK_CI(qi);
      constexpr int t = qq / (TY * TZ), u = (qq / TZ) % TY, v = qq % TZ;
      const float e1 = __ldg(EQ + e0 + qq);
      const float ev = ((t + u + v) & 1) ? -e1 : e1;
      sfor<NHAB>([&](auto pi) {
        constexpr int p = FK_CI(pi);
        constexpr TUV h = ct_hvec(p);
        Y[p * NCD + kc] = fmaf(ev, R[ct_hidx(h.t + t, h.u + u, h.v + v)], Y[p * NCD + kc]);
      });
    });
  });
}

// FP32 bra transform ERI[ab][cd] += sum_p E^{ab}_p Y[p][cd], each element
// handed to put(index, value) (accumulation left to the caller).
template <int LA, int LB, int LC, int LD, class Put>
__device__ __forceinline__ void bra_f32(const float *__restrict__ EP,
                                        const float (&Y)[nherm(LA + LB) * ncart(LC) * ncart(LD)], Put &&put) {
  constexpr int NB = ncart(LB), NAB = ncart(LA) * NB, NCD = ncart(LC) * ncart(LD);
  sfor<NAB>([&](auto kai) {
    constexpr int ka = FK_CI(kai);
    constexpr TUV c = ct_cart(LA, ka / NB), d = ct_cart(LB, ka % NB);
    constexpr int TY = c.u + d.u + 1, TZ = c.v + d.v + 1, NQ = (c.t + d.t + 1) * TY * TZ;
    constexpr int e0 = ct_eoff(LA, LB, ka);
    sfor<NCD>([&](auto kci) {
      constexpr int kc = FK_CI(kci);
      float s = 0.0f;
      sfor<NQ>([&](auto qi) {
        constexpr int qq = FK_CI(qi);
        constexpr int t = qq / (TY * TZ), u = (qq / TZ) % TY, v = qq % TZ;
        s = fmaf(__ldg(EP + e0 + qq), Y[ct_hidx(t, u, v) * NCD + kc], s);
      });
      put(ka * NCD + kc, s);
    });
  });
}

// The FP32 part of an FP64 quartet in mixed precision: every primitive quartet
// that passes the primitive screen but whose bound is below the FP32 cutoff
// (prim_fp32), i.e. exactly those the FP64 loops of quartet_reg_f64 left out.
// Per bra primitive the FP32 contributions are summed in FP32 and each
// element is handed to add(index, value) once.
template <int LA, int LB, int LC, int LD, class Add>
__device__ __forceinline__ void prim_tail_f32(const KArgs &a, const MolView &mv, const PrimScreen &ps, int P, int Q,
                                              int sA, int sC, Add &&add) {
  constexpr int NCD = ncart(LC) * ncart(LD), NHAB = nherm(LA + LB);
  const DevPairs &dp = a.dp;
  const float *ha = dp.shl + 6 * sA, *hc = dp.shl + 6 * sC;
  const float ACx = (ha[0] - hc[0]) + (ha[3] - hc[3]);
  const float ACy = (ha[1] - hc[1]) + (ha[4] - hc[4]);
  const float ACz = (ha[2] - hc[2]) + (ha[5] - hc[5]);
  const int2 pb = dp.prim[P], pk = dp.prim[Q];
  const int kend = pk.x + pk.y;
  for (int ip = pb.x; ip < pb.x + pb.y; ++ip) {
    if (prim_skip(a, mv, ps, ip, pk.x)) break;
    int j0 = pk.x;
    while (j0 < kend && !prim_fp32(a, ps, ip, j0)) ++j0;
    if (j0 == kend || prim_skip(a, mv, ps, ip, j0)) continue;
    const float4 PA = dp.paf[ip];
    float Y[NHAB * NCD];
    sfor<NHAB * NCD>([&](auto i) { Y[FK_CI(i)] = 0.0f; });
    for (int jq = j0; jq < kend; ++jq) {
      if (prim_skip(a, mv, ps, ip, jq)) break;
      prim_f32_ket<LA, LB, LC, LD>(a, PA, jq, ACx, ACy, ACz, Y);
    }
    bra_f32<LA, LB, LC, LD>(dp.Ef + dp.eoff[ip], Y, add);
  }
}

template <int LA, int LB, int LC, int LD, bool MIXED>
__device__ __forceinline__ void quartet_reg_f64(const KArgs &a, const MolView &mv, int P, int Q, int sA, int sB,
                                                int sC, int sD, double *eri_col) {
  constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  constexpr int NAB = NA * NB, NCD = NC * ND;
  constexpr int LAB = LA + LB, L = LA + LB + LC + LD;
  constexpr int NHAB = nherm(LAB), NHL = nherm(L);
  constexpr bool SM = reg_eri_in_smem<LA, LB, LC, LD>();
  const DevPairs &dp = a.dp;

  double eri_r[SM ? 1 : NAB * NCD];
  const int bs = blockDim.x;
  auto eri_at = [&](int i) -> double & {
    if constexpr (SM)
      return eri_col[i * bs];
    else
      return eri_r[i];
  };
  sfor<NAB * NCD>([&](auto i) { eri_at(FK_CI(i)) = 0.0; });
  const int2 pb = dp.prim[P], pk = dp.prim[Q];
  const PrimScreen ps = prim_screen<MIXED>(a, mv, sA, sB, sC, sD);
  for (int ip = pb.x; ip < pb.x + pb.y; ++ip) {
    if (prim_skip(a, mv, ps, ip, pk.x)) break;  // weaker bra primitives follow
    if (MIXED && prim_fp32(a, ps, ip, pk.x)) break;  // the rest is FP32 work (below)
    const PZ P4 = dp.pz[ip];
    const float4 Pf = dp.pf[ip];
    double Y[NHAB * NCD];
    sfor<NHAB * NCD>([&](auto i) { Y[FK_CI(i)] = 0.0; });
    for (int jq = pk.x; jq < pk.x + pk.y; ++jq) {
      if (prim_skip(a, mv, ps, ip, jq)) break;  // weaker ket primitives follow
      if (MIXED && prim_fp32(a, ps, ip, jq)) break;
      const PrimQuartet q = prim_quartet(P4, Pf, dp.pz[jq], dp.pf[jq]);
      double F[L + 1];
      boys_seeds<L>(a.boys, q, F, a.boysf);
      double R[NHL];
      hermite_r_reg<L, double>(F, q.X, q.Y, q.Z, R);
      // ket transform: Y[p][cd] += sum_q (-1)^{|q|} E^{cd}_q R_{p+q}
      const double *__restrict__ EQ = dp.E + dp.eoff[jq];
      sfor<NCD>([&](auto kci) {
        constexpr int kc = FK_CI(kci);
        constexpr TUV c = ct_cart(LC, kc / ND), d = ct_cart(LD, kc % ND);
        constexpr int TY = c.u + d.u + 1, TZ = c.v + d.v + 1, NQ = (c.t + d.t + 1) * TY * TZ;
        constexpr int e0 = ct_eoff(LC, LD, kc);
        sfor<NQ>([&](auto qi) {
          constexpr int qq = FK_CI(qi);
          constexpr int t = qq / (TY * TZ), u = (qq / TZ) % TY, v = qq % TZ;
          const double e1 = __ldg(EQ + e0 + qq);
          const double ev = ((t + u + v) & 1) ? -e1 : e1;
          sfor<NHAB>([&](auto pi) {
            constexpr int p = FK_CI(pi);
            constexpr TUV h = ct_hvec(p);
            Y[p * NCD + kc] = fma(ev, R[ct_hidx(h.t + t, h.u + u, h.v + v)], Y[p * NCD + kc]);
          });
        });
      });
    }
    // bra transform: ERI[ab][cd] += sum_p E^{ab}_p Y[p][cd]
    const double *__restrict__ EP = dp.E + dp.eoff[ip];
    sfor<NAB>([&](auto kai) {
      constexpr int ka = FK_CI(kai);
      constexpr TUV c = ct_cart(LA, ka / NB), d = ct_cart(LB, ka % NB);
      constexpr int TY = c.u + d.u + 1, TZ = c.v + d.v + 1, NQ = (c.t + d.t + 1) * TY * TZ;
      constexpr int e0 = ct_eoff(LA, LB, ka);
      sfor<NQ>([&](auto qi) {
        constexpr int qq = FK_CI(qi);
        constexpr int t = qq / (TY * TZ), u = (qq / TZ) % TY, v = qq % TZ;
        const double ev = __ldg(EP + e0 + qq);
        sfor<NCD>([&](auto kci) {
          constexpr int kc = FK_CI(kci);
          eri_at(ka * NCD + kc) = fma(ev, Y[ct_hidx(t, u, v) * NCD + kc], eri_at(ka * NCD + kc));
        });
      });
    });
  }

  // mixed precision: the primitive quartets below the cutoff, in FP32
  if constexpr (MIXED) {
    if (ps.c32 > 0.0f) prim_tail_f32<LA, LB, LC, LD>(a, mv, ps, P, Q, sA, sC, [&](int i, float v) {
      eri_at(i) += f2d_any(v);
    });
  }

  // digestion into the six J/K blocks (8-fold symmetry, Sec. 2.3 / 3.2)
  double fac = 1.0;
  if (sA == sB) fac *= 0.5;
  if (sC == sD) fac *= 0.5;
  if (P == Q) fac *= 0.5;
  const double fac2 = 2.0 * fac;
  const int N = mv.N;
  const int fa = dp.sbf[sA], fb = dp.sbf[sB], fc = dp.sbf[sC], fd = dp.sbf[sD];
  const double *__restrict__ Dm = mv.D;
  double *__restrict__ Jm = mv.J;
  double *__restrict__ Km = mv.K;
  auto E4 = [&](int ia, int ib, int ic, int id) -> double { return eri_at((ia * NB + ib) * NCD + ic * ND + id); };
  auto Dv = [&](int r, int c) -> double { return __ldg(Dm + (size_t)r * N + c); };
  if (!MIXED || (a.parts & 1)) {
  sfor<NAB>([&](auto k) {  // J_ab += (ab|cd) D_cd
    constexpr int ia = FK_CI(k) / NB, ib = FK_CI(k) % NB;
    double s = 0.0;
    sfor<NCD>([&](auto m) { s = fma(E4(ia, ib, FK_CI(m) / ND, FK_CI(m) % ND), Dv(fc + FK_CI(m) / ND, fd + FK_CI(m) % ND), s); });
    atomicAdd(Jm + (size_t)(fa + ia) * N + fb + ib, fac2 * s);
  });
  sfor<NCD>([&](auto k) {  // J_cd += (ab|cd) D_ab
    constexpr int ic = FK_CI(k) / ND, id = FK_CI(k) % ND;
    double s = 0.0;
    sfor<NAB>([&](auto m) { s = fma(E4(FK_CI(m) / NB, FK_CI(m) % NB, ic, id), Dv(fa + FK_CI(m) / NB, fb + FK_CI(m) % NB), s); });
    atomicAdd(Jm + (size_t)(fc + ic) * N + fd + id, fac2 * s);
  });
  }
  if (MIXED && !(a.parts & 2)) return;
  sfor<NA * NC>([&](auto k) {  // K_ac += (ab|cd) D_bd
    constexpr int ia = FK_CI(k) / NC, ic = FK_CI(k) % NC;
    double s = 0.0;
    sfor<NB * ND>([&](auto m) { s = fma(E4(ia, FK_CI(m) / ND, ic, FK_CI(m) % ND), Dv(fb + FK_CI(m) / ND, fd + FK_CI(m) % ND), s); });
    atomicAdd(Km + (size_t)(fa + ia) * N + fc + ic, fac * s);
  });
  sfor<NA * ND>([&](auto k) {  // K_ad += (ab|cd) D_bc
    constexpr int ia = FK_CI(k) / ND, id = FK_CI(k) % ND;
    double s = 0.0;
    sfor<NB * NC>([&](auto m) { s = fma(E4(ia, FK_CI(m) / NC, FK_CI(m) % NC, id), Dv(fb + FK_CI(m) / NC, fc + FK_CI(m) % NC), s); });
    atomicAdd(Km + (size_t)(fa + ia) * N + fd + id, fac * s);
  });
  sfor<NB * NC>([&](auto k) {  // K_bc += (ab|cd) D_ad
    constexpr int ib = FK_CI(k) / NC, ic = FK_CI(k) % NC;
    double s = 0.0;
    sfor<NA * ND>([&](auto m) { s = fma(E4(FK_CI(m) / ND, ib, ic, FK_CI(m) % ND), Dv(fa + FK_CI(m) / ND, fd + FK_CI(m) % ND), s); });
    atomicAdd(Km + (size_t)(fb + ib) * N + fc + ic, fac * s);
  });
  sfor<NB * ND>([&](auto k) {  // K_bd += (ab|cd) D_ac
    constexpr int ib = FK_CI(k) / ND, id = FK_CI(k) % ND;
    double s = 0.0;
    sfor<NA * NC>([&](auto m) { s = fma(E4(FK_CI(m) / NC, ib, FK_CI(m) % NC, id), Dv(fa + FK_CI(m) / NC, fc + FK_CI(m) % NC), s); });
    atomicAdd(Km + (size_t)(fb + ib) * N + fd + id, fac * s);
  });
}

// The same quartet in FP32 (mixed-precision path, quartets whose
// density-weighted bound is below the FP32 cutoff): FP32 Boys table, Hermite
// recursion, transforms and digestion; centres are taken relative to the
// pair's first shell so that P - Q keeps its precision; each digested J/K
// element is converted exactly to FP64 and accumulated in FP64.
// Classes with total L >= 5 (FP32 quartets only, k_reg32) keep the FP32
// contracted-ERI accumulator in per-thread shared memory, [element][thread].
template <int LA, int LB, int LC, int LD>
__host__ __device__ constexpr bool reg32_eri_in_smem() {
  return LA + LB + LC + LD >= 5;
}
template <int LA, int LB, int LC, int LD>
__host__ __device__ constexpr int reg32_smem_bytes(int threads) {
  return reg32_eri_in_smem<LA, LB, LC, LD>() ? ncart(LA) * ncart(LB) * ncart(LC) * ncart(LD) * threads * 4 : 0;
}

template <int LA, int LB, int LC, int LD>
__device__ __forceinline__ void quartet_reg_f32(const KArgs &a, const MolView &mv, int P, int Q, int sA, int sB,
                                                int sC, int sD, float *eri_col = nullptr) {
  constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  constexpr int NAB = NA * NB, NCD = NC * ND;
  constexpr int LAB = LA + LB, L = LA + LB + LC + LD;
  constexpr int NHAB = nherm(LAB), NHL = nherm(L);
  constexpr bool SM = reg32_eri_in_smem<LA, LB, LC, LD>();
  const DevPairs &dp = a.dp;
  // A - C from hi/lo FP32 parts: the hi difference rounds once relative to
  // |A - C| itself, the lo parts restore the bits the hi parts dropped
  const float *ha = dp.shl + 6 * sA, *hc = dp.shl + 6 * sC;
  const float ACx = (ha[0] - hc[0]) + (ha[3] - hc[3]);
  const float ACy = (ha[1] - hc[1]) + (ha[4] - hc[4]);
  const float ACz = (ha[2] - hc[2]) + (ha[5] - hc[5]);
  float eri_r[SM ? 1 : NAB * NCD];
  const int bs = blockDim.x;
  auto eri = [&](int i) -> float & {
    if constexpr (SM)
      return eri_col[i * bs];
    else
      return eri_r[i];
  };
  sfor<NAB * NCD>([&](auto i) { eri(FK_CI(i)) = 0.0f; });
  const int2 pb = dp.prim[P], pk = dp.prim[Q];
  const PrimScreen ps = prim_screen(a, mv, sA, sB, sC, sD);
  for (int ip = pb.x; ip < pb.x + pb.y; ++ip) {
    if (prim_skip(a, mv, ps, ip, pk.x)) break;
    const float4 PA = dp.paf[ip];
    float Y[NHAB * NCD];
    sfor<NHAB * NCD>([&](auto i) { Y[FK_CI(i)] = 0.0f; });
    for (int jq = pk.x; jq < pk.x + pk.y; ++jq) {
      if (prim_skip(a, mv, ps, ip, jq)) break;
      const float4 QC = dp.paf[jq];
      const float X = PA.x - QC.x + ACx, Yd = PA.y - QC.y + ACy, Z = PA.z - QC.z + ACz;
      const float rs = rsqrtf(PA.w + QC.w);
      const float alpha = (PA.w * QC.w) * (rs * rs);
      const float T = alpha * fmaf(X, X, fmaf(Yd, Yd, Z * Z));
      float F[L + 1];
      boys_seeds_f32<L>(a.boysf, T, rs, -2.0f * alpha, F);
      float R[NHL];
      hermite_r_reg<L, float>(F, X, Yd, Z, R);
      const float *__restrict__ EQ = dp.Ef + dp.eoff[jq];
      sfor<NCD>([&](auto kci) {
        constexpr int kc = FK_CI(kci);
        constexpr TUV c = ct_cart(LC, kc / ND), d = ct_cart(LD, kc % ND);
        constexpr int TY = c.u + d.u + 1, TZ = c.v + d.v + 1, NQ = (c.t + d.t + 1) * TY * TZ;
        constexpr int e0 = ct_eoff(LC, LD, kc);
        sfor<NQ>([&](auto qi) {
          constexpr int qq = FK_CI(qi);
          constexpr int t = qq / (TY * TZ), u = (qq / TZ) % TY, v = qq % TZ;
          const float e1 = __ldg(EQ + e0 + qq);
          const float ev = ((t + u + v) & 1) ? -e1 : e1;
          sfor<NHAB>([&](auto pi) {
            constexpr int p = FK_CI(pi);
            constexpr TUV h = ct_hvec(p);
            Y[p * NCD + kc] = fmaf(ev, R[ct_hidx(h.t + t, h.u + u, h.v + v)], Y[p * NCD + kc]);
          });
        });
      });
    }
    const float *__restrict__ EP = dp.Ef + dp.eoff[ip];
    sfor<NAB>([&](auto kai) {
      constexpr int ka = FK_CI(kai);
      constexpr TUV c = ct_cart(LA, ka / NB), d = ct_cart(LB, ka % NB);
      constexpr int TY = c.u + d.u + 1, TZ = c.v + d.v + 1, NQ = (c.t + d.t + 1) * TY * TZ;
      constexpr int e0 = ct_eoff(LA, LB, ka);
      sfor<NQ>([&](auto qi) {
        constexpr int qq = FK_CI(qi);
        constexpr int t = qq / (TY * TZ), u = (qq / TZ) % TY, v = qq % TZ;
        const float ev = __ldg(EP + e0 + qq);
        sfor<NCD>([&](auto kci) {
          constexpr int kc = FK_CI(kci);
          eri(ka * NCD + kc) = fmaf(ev, Y[ct_hidx(t, u, v) * NCD + kc], eri(ka * NCD + kc));
        });
      });
    });
  }
  float fac = 1.0f;
  if (sA == sB) fac *= 0.5f;
  if (sC == sD) fac *= 0.5f;
  if (P == Q) fac *= 0.5f;
  const float fac2 = 2.0f * fac;
  const int N = mv.N;
  const int fa = dp.sbf[sA], fb = dp.sbf[sB], fc = dp.sbf[sC], fd = dp.sbf[sD];
  const float *__restrict__ Dm = mv.Df;
  double *__restrict__ Jm = mv.J;
  double *__restrict__ Km = mv.K;
  auto E4 = [&](int ia, int ib, int ic, int id) -> float { return eri((ia * NB + ib) * NCD + ic * ND + id); };
  auto Dv = [&](int r, int c) -> float { return __ldg(Dm + (size_t)r * N + c); };
  if (a.parts & 1) {
  sfor<NAB>([&](auto k) {
    constexpr int ia = FK_CI(k) / NB, ib = FK_CI(k) % NB;
    float s = 0.0f;
    sfor<NCD>([&](auto m) { s = fmaf(E4(ia, ib, FK_CI(m) / ND, FK_CI(m) % ND), Dv(fc + FK_CI(m) / ND, fd + FK_CI(m) % ND), s); });
    atomicAdd(Jm + (size_t)(fa + ia) * N + fb + ib, f2d_any(fac2 * s));
  });
  sfor<NCD>([&](auto k) {
    constexpr int ic = FK_CI(k) / ND, id = FK_CI(k) % ND;
    float s = 0.0f;
    sfor<NAB>([&](auto m) { s = fmaf(E4(FK_CI(m) / NB, FK_CI(m) % NB, ic, id), Dv(fa + FK_CI(m) / NB, fb + FK_CI(m) % NB), s); });
    atomicAdd(Jm + (size_t)(fc + ic) * N + fd + id, f2d_any(fac2 * s));
  });
  }
  if (!(a.parts & 2)) return;
  sfor<NA * NC>([&](auto k) {
    constexpr int ia = FK_CI(k) / NC, ic = FK_CI(k) % NC;
    float s = 0.0f;
    sfor<NB * ND>([&](auto m) { s = fmaf(E4(ia, FK_CI(m) / ND, ic, FK_CI(m) % ND), Dv(fb + FK_CI(m) / ND, fd + FK_CI(m) % ND), s); });
    atomicAdd(Km + (size_t)(fa + ia) * N + fc + ic, f2d_any(fac * s));
  });
  sfor<NA * ND>([&](auto k) {
    constexpr int ia = FK_CI(k) / ND, id = FK_CI(k) % ND;
    float s = 0.0f;
    sfor<NB * NC>([&](auto m) { s = fmaf(E4(ia, FK_CI(m) / NC, FK_CI(m) % NC, id), Dv(fb + FK_CI(m) / NC, fc + FK_CI(m) % NC), s); });
    atomicAdd(Km + (size_t)(fa + ia) * N + fd + id, f2d_any(fac * s));
  });
  sfor<NB * NC>([&](auto k) {
    constexpr int ib = FK_CI(k) / NC, ic = FK_CI(k) % NC;
    float s = 0.0f;
    sfor<NA * ND>([&](auto m) { s = fmaf(E4(FK_CI(m) / ND, ib, ic, FK_CI(m) % ND), Dv(fa + FK_CI(m) / ND, fd + FK_CI(m) % ND), s); });
    atomicAdd(Km + (size_t)(fb + ib) * N + fc + ic, f2d_any(fac * s));
  });
  sfor<NB * ND>([&](auto k) {
    constexpr int ib = FK_CI(k) / ND, id = FK_CI(k) % ND;
    float s = 0.0f;
    sfor<NA * NC>([&](auto m) { s = fmaf(E4(FK_CI(m) / NC, ib, FK_CI(m) % NC, id), Dv(fa + FK_CI(m) / NC, fc + FK_CI(m) % NC), s); });
    atomicAdd(Km + (size_t)(fb + ib) * N + fd + id, f2d_any(fac * s));
  });
}

// Warp-level work queue: a unit's kets are screened 32 at a time and the
// surviving (bra, ket) pairs appended to an FP64 or an FP32 queue (ballot +
// prefix popcount); each full queue is drained 32 quartets at a time, so every
// batch runs one precision with all lanes busy and screened-out quartets cost
// no lane time.  The queues carry over from one unit to the next (all units
// of a launch are of one class pair), so a warp leaves a partly filled batch
// only once, after its last unit.
template <int LA, int LB, int LC, int LD, bool MIXED, bool F32>
__device__ __forceinline__ void drain_reg(const KArgs &a, int *qp, int *qq, int &n, double *eri_col, int lane) {
  const int m = n < 32 ? n : 32;
  if (lane < m) {
    const int P = qp[lane], Q = qq[lane];
    const int2 ab = a.dp.ab[P], cd = a.dp.ab[Q];
    const MolView mv = mol_view(a, ab.x);
    if constexpr (F32)
      quartet_reg_f32<LA, LB, LC, LD>(a, mv, P, Q, ab.x, ab.y, cd.x, cd.y);
    else
      quartet_reg_f64<LA, LB, LC, LD, MIXED>(a, mv, P, Q, ab.x, ab.y, cd.x, cd.y, eri_col);
  }
  __syncwarp();
  // move the rest (< 32 entries) forward
  const bool mv_ = lane + 32 < n;
  const int rp = mv_ ? qp[lane + 32] : 0, rq = mv_ ? qq[lane + 32] : 0;
  __syncwarp();
  if (mv_) {
    qp[lane] = rp;
    qq[lane] = rq;
  }
  n -= m;
  __syncwarp();
}

// MIXED = false: the lean FP64 fused J+K build (no FP32 code, exact test
// only); true: every feature -- mixed precision (FP32 quartets below the
// cutoff, FP32 primitive tails above it), J-only / K-only builds and the
// decay-bound exchange test.  One loop screens a 32-ket chunk per pass and
// drains whichever queue holds a full batch (every queue at the end), so
// each quartet body is inlined once.
template <int LA, int LB, int LC, int LD, bool MIXED>
__global__ void __launch_bounds__(128) k_reg(KArgs a) {
  extern __shared__ __align__(16) double reg_smem[];
  constexpr int NQ = MIXED ? 2 : 1;  // FP64 queue, FP32 queue
  __shared__ int queues[4][NQ][2][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *eri_col = reg_smem + threadIdx.x;
  int *p64 = queues[warp][0][0], *q64 = queues[warp][0][1];
  int *p32 = queues[warp][NQ - 1][0], *q32 = queues[warp][NQ - 1][1];
  const unsigned lt = (1u << lane) - 1u;
  int n64 = 0, n32 = 0;
  bool more = true;  // units left to screen
  int P = 0, c = 0, k1 = 0;
  for (;;) {
    if (more && c >= k1) {
      const int u = next_unit(a.counter, lane);
      if (u < a.nunits) {
        const Unit un = a.units[u];
        P = un.bra;
        c = un.k0;
        k1 = un.k1;
      } else {
        more = false;
      }
    }
    if (more) {
      const int2 ab = a.dp.ab[P];
      const int Q = c + lane;
      float b = -1.0f;
      if (Q < k1) {
        const MolView mv = mol_view(a, ab.x);
        const int2 cd = a.dp.ab[Q];
        b = quartet_bound<MIXED>(a, mv, ab.x, ab.y, cd.x, cd.y, P, Q);
      }
      c += 32;
      const bool is32 = MIXED && b >= 0.0f && b < a.fp32_cutoff_f, is64 = b >= 0.0f && !is32;
      const unsigned m64 = __ballot_sync(0xffffffffu, is64), m32 = __ballot_sync(0xffffffffu, is32);
      if (is64) {
        const int k = n64 + __popc(m64 & lt);
        p64[k] = P;
        q64[k] = Q;
      }
      if (is32) {
        const int k = n32 + __popc(m32 & lt);
        p32[k] = P;
        q32[k] = Q;
      }
      n64 += __popc(m64);
      n32 += __popc(m32);
      __syncwarp();
    }
    if (n64 >= 32 || (!more && n64 > 0)) drain_reg<LA, LB, LC, LD, MIXED, false>(a, p64, q64, n64, eri_col, lane);
    if constexpr (MIXED) {
      if (n32 >= 32 || (!more && n32 > 0)) drain_reg<LA, LB, LC, LD, MIXED, true>(a, p32, q32, n32, eri_col, lane);
    }
    if (!more && n64 == 0 && n32 == 0) break;
  }
}

// FP32 quartets of a class pair with total L = 5 (the FP32 part of a mixed
// group tier; its FP64 quartets run on the group kernel): one thread per
// quartet with compile-time loops, the FP32 ERI accumulator in per-thread
// shared memory.  Same warp queue as k_reg, FP32 quartets only.
template <int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(128) k_reg32(KArgs a) {
  extern __shared__ __align__(16) float reg32_smem[];
  __shared__ int queues[4][2][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *eri_col = reg32_smem + threadIdx.x;
  int *qp = queues[warp][0], *qq = queues[warp][1];
  const unsigned lt = (1u << lane) - 1u;
  auto drain = [&](int n) {
    if (lane < n) {
      const int P = qp[lane], Q = qq[lane];
      const int2 ab = a.dp.ab[P], cd = a.dp.ab[Q];
      const MolView mv = mol_view(a, ab.x);
      quartet_reg_f32<LA, LB, LC, LD>(a, mv, P, Q, ab.x, ab.y, cd.x, cd.y, eri_col);
    }
  };
  int n32 = 0;
  for (;;) {
    const int u = next_unit(a.counter, lane);
    if (u >= a.nunits) break;
    const Unit un = a.units[u];
    const int P = un.bra;
    const int2 ab = a.dp.ab[P];
    const MolView mv = mol_view(a, ab.x);
    for (int c = un.k0; c < un.k1; c += 32) {
      const int Q = c + lane;
      float b = -1.0f;
      if (Q < un.k1) {
        const int2 cd = a.dp.ab[Q];
        b = quartet_bound(a, mv, ab.x, ab.y, cd.x, cd.y, P, Q);
      }
      const bool is32 = b >= 0.0f && b < a.fp32_cutoff_f;
      const unsigned m32 = __ballot_sync(0xffffffffu, is32);
      if (is32) {
        const int k = n32 + __popc(m32 & lt);
        qp[k] = P;
        qq[k] = Q;
      }
      n32 += __popc(m32);
      __syncwarp();
      if (n32 >= 32) {
        drain(32);
        __syncwarp();
        const bool mv_ = lane + 32 < n32;
        const int rp = mv_ ? qp[lane + 32] : 0, rq = mv_ ? qq[lane + 32] : 0;
        __syncwarp();
        if (mv_) {
          qp[lane] = rp;
          qq[lane] = rq;
        }
        n32 -= 32;
        __syncwarp();
      }
    }
  }
  drain(n32);
}

// (bra class, ket class) pairs served by register kernels: total L <= 4
__host__ __device__ constexpr bool reg_class_pair(int cb, int ck) {
  constexpr int Lc[NCLASS] = {0, 1, 2, 2, 3, 4, 3, 4, 5, 6};
  return cb >= 0 && ck >= 0 && cb < NCLASS && ck < NCLASS && Lc[cb] + Lc[ck] <= 4;
}

}  // namespace fk
