// GB300 (sm_103a) kernels of the J/K build.
//
// Integral scheme: McMurchie-Davidson (arXiv:2407.21445 Sec. 4.1, Eqs. MD
// def, EabP def1-3): a primitive quartet is
//   [ab|cd] = sum_p sum_q E^{ab}_p (-1)^{|q|} R_{p+q} E^{cd}_q ,
// R_{tuv} from the Hermite recursion R^{(n)}_{t+1,u,v} = t R^{(n+1)}_{t-1,u,v}
// + X_PQ R^{(n+1)}_{tuv} seeded by R^{(n)}_{000} = pref (-2 alpha)^n F_n(T),
// pref = U_P U_Q 2 sqrt(alpha/pi), alpha = zeta eta / (zeta + eta),
// T = alpha |P-Q|^2 (the paper's garbled seed read this way).
//
// Work decomposition: a "group" of G lanes (G = 1..32, a power of two, chosen
// per class pair) owns one contracted shell quartet (ab|cd) at a time.  For
// each bra primitive pair it accumulates over the ket primitive pairs the
// half-transformed Y[p][cd] = sum_q (-1)^{|q|} E^{cd}_q R_{p+q}, then applies
// the bra transform ERI[ab][cd] += sum_p E^{ab}_p Y[p][cd]; the contracted
// ERIs are then digested with the density into the six J/K blocks of the
// 8-fold permutational symmetry (Sec. 2.3, Sec. 3.2 "six Fock matrix
// blocks").  The intermediates live in a per-group shared-memory scratch.
// Groups of one warp take consecutive ket pairs of one bra pair from a work
// unit; warps pull units from a global counter (persistent grid).
//
// GB300 executes FP64 at 1/64 of the FP32 rate, so the kernels are bound by
// the FP64 pipe; index arithmetic, shared-memory traffic and FP32 work are
// comparatively free and are spent freely to keep FP64 lanes busy.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "device_common.cuh"
#include "kargs.cuh"
#include "reg_dispatch.h"

namespace fk {

__device__ int g_status = 0;  // sticky device status word (fock_status)

// Diagnostic bounds checks (compiled in with -DFOCK_BOUNDS_CHECK): a failed
// check records its site and the offending value in g_bounds and skips the
// quartet instead of touching memory.
__device__ long long g_bounds[2] = {0, 0};
#ifdef FOCK_BOUNDS_CHECK
#define FK_CHECK(cond, site, val)                                          \
  do {                                                                     \
    if (!(cond)) {                                                         \
      if (atomicCAS((unsigned long long *)&g_bounds[0], 0ull, (unsigned long long)(site)) == 0ull) \
        g_bounds[1] = (long long)(val);                                    \
      return;                                                              \
    }                                                                      \
  } while (0)
#else
#define FK_CHECK(cond, site, val) \
  do {                            \
  } while (0)
#endif

static double *s_boys[64];
static float *s_boysf[64];
static ClassTables *s_tabs[64];



static_assert(sizeof(ClassTables) % 16 == 0, "table copy uses whole 4-byte words");
constexpr int TAB_BYTES = (int)sizeof(ClassTables);

// Scratch stride (in doubles) of a group running the FP32 body: its
// intermediates take half the bytes; kept odd for the shared-memory banks.
__host__ __device__ constexpr int fp32_stride(int stride) { return ((stride + 1) / 2) | 1; }

__device__ __forceinline__ void group_sync(unsigned mask, int G) {
  if (G > 1) __syncwarp(mask);
}

// R^{(0)}_{tuv}, t+u+v <= L, into the returned buffer (one of R0/R1).
// F must hold base values pref (-2alpha)^n F_n(T), n = 0..L; R0[0] = F[L].
__constant__ double c_small[16] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15};
__constant__ float c_smallf[16] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15};

// x with its sign flipped when s == 1 (integer units only)
__device__ __forceinline__ double neg_if(double x, int s) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)s << 63));
}
__device__ __forceinline__ float neg_if(float x, int s) {
  return __int_as_float(__float_as_int(x) ^ (s << 31));
}

template <class Real>
__device__ __forceinline__ Real small_int(int i) {
  if constexpr (sizeof(Real) == 8)
    return c_small[i];
  else
    return c_smallf[i];
}

template <int G, class Real>
__device__ __forceinline__ Real *hermite_r(const ClassTables &ct, int L, Real X, Real Y, Real Z, const Real *F,
                                           Real *R0, Real *R1, int gl, unsigned gmask) {
  Real *cur = R0, *nxt = R1;
  for (int n = L - 1; n >= 0; --n) {
    int cnt = nherm(L - n);
    for (int e = gl; e < cnt; e += G) {
      Real v;
      if (e == 0) {
        v = F[n];
      } else {
        int t = ct.hvec[e][0], u = ct.hvec[e][1], w = ct.hvec[e][2];
        if (t > 0) {
          v = X * cur[hidx(t - 1, u, w)];
          if (t > 1) v = fma(small_int<Real>(t - 1), cur[hidx(t - 2, u, w)], v);
        } else if (u > 0) {
          v = Y * cur[hidx(t, u - 1, w)];
          if (u > 1) v = fma(small_int<Real>(u - 1), cur[hidx(t, u - 2, w)], v);
        } else {
          v = Z * cur[hidx(t, u, w - 1)];
          if (w > 1) v = fma(small_int<Real>(w - 1), cur[hidx(t, u, w - 2)], v);
        }
      }
      nxt[e] = v;
    }
    group_sync(gmask, G);
    Real *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  return cur;
}

// FP32 seeds for the group kernel (lanes over m), R0[0] = F[L].
template <int G>
__device__ __forceinline__ void boys_seeds_rt_f32(const float *__restrict__ tab, float T, float pref, float m2a, int L,
                                                  float *F, float *R0, int gl) {
  for (int m = gl; m <= L; m += G) {
    float f;
    if (T < (float)BOYS_TMAX) {
      const int gi = __float2int_rn(T * (float)BOYS_INVH);
      const float x = (float)gi * (float)BOYS_H - T;
      const float4 *c = reinterpret_cast<const float4 *>(tab + ((size_t)gi * (LTOT + 1) + m) * BOYS_TAYLOR);
      const float4 c03 = __ldg(c);
      const float2 c45 = __ldg(reinterpret_cast<const float2 *>(c + 1));
      f = fmaf(c45.y, x, c45.x);
      f = fmaf(f, x, c03.w);
      f = fmaf(f, x, c03.z);
      f = fmaf(f, x, c03.y);
      f = fmaf(f, x, c03.x);
    } else {
      const float rt = rsqrtf(T), it = rt * rt;
      f = 0.886226925452758f * rt;
      for (int k = 1; k <= m; ++k) f *= ((float)k - 0.5f) * it;
    }
    float c = pref;
    for (int k = 0; k < m; ++k) c *= m2a;
    F[m] = f * c;
    if (m == L) R0[0] = F[m];
  }
}

// Ket transform of one primitive quartet, accumulated over ket primitives:
// Yh[p][cd] += sum_q (-1)^{|q|} E^{cd}_q R_{p+q}.  Elements are walked in
// ket-component-major order, so the lanes of a group work on the same ket
// component (same Hermite box, same trip counts) for consecutive bra
// Hermite indices; two independent accumulation chains (even / odd v).
template <int G, class Real>
__device__ __forceinline__ void ket_transform(const ClassTables &ct, const Real *EQ, const Real *R, Real *Yh,
                                              int nhab, int ncd, int nd, int lc, int ld, int ck, int gl) {
  for (int it = gl; it < nhab * ncd; it += G) {
    const int kc = it / nhab, ph = it - kc * nhab;
    const int tp = ct.hvec[ph][0], up = ct.hvec[ph][1], vp = ct.hvec[ph][2];
    const int ic = kc / nd, id = kc - ic * nd;
    const uint8_t *cc = ct.comp[lc][ic], *dd = ct.comp[ld][id];
    const int Tx = cc[0] + dd[0], Ty = cc[1] + dd[1], Tz = cc[2] + dd[2];
    const Real *Eq = EQ + ct.eoff[ck][kc];
    const int yi = ph * ncd + kc;  // Yh layout: [bra Hermite index][ket component]
    Real acc0 = Yh[yi], acc1 = Real(0);
    int e = 0;
    for (int t = 0; t <= Tx; ++t)
      for (int u = 0; u <= Ty; ++u) {
        const int s = (t + u) & 1;  // (-1)^(t+u+v): s for even v, flipped for odd v
        int v = 0;
        for (; v < Tz; v += 2, e += 2) {
          const Real r0 = R[hidx(tp + t, up + u, vp + v)], r1 = R[hidx(tp + t, up + u, vp + v + 1)];
          acc0 = fma(neg_if(Eq[e], s), r0, acc0);
          acc1 = fma(neg_if(Eq[e + 1], s ^ 1), r1, acc1);
        }
        if (v == Tz) {
          acc0 = fma(neg_if(Eq[e], s), R[hidx(tp + t, up + u, vp + v)], acc0);
          ++e;
        }
      }
    Yh[yi] = acc0 + acc1;
  }
}

// Bra transform ERI[ab][cd] += sum_p E^{ab}_p Yh[p][cd] (two accumulation
// chains, even / odd v).
template <int G, class Real>
__device__ __forceinline__ void bra_transform(const ClassTables &ct, const Real *EP, const Real *Yh, Real *eri, int nab,
                                              int ncd, int nb, int la, int lb, int cb, int gl) {
  for (int it = gl; it < nab * ncd; it += G) {
    const int ka = it / ncd, kc = it - ka * ncd;
    const int ia = ka / nb, ib = ka - ia * nb;
    const uint8_t *ac = ct.comp[la][ia], *bc = ct.comp[lb][ib];
    const int Tx = ac[0] + bc[0], Ty = ac[1] + bc[1], Tz = ac[2] + bc[2];
    const Real *Ep = EP + ct.eoff[cb][ka];
    Real acc0 = eri[it], acc1 = Real(0);
    int e = 0;
    for (int t = 0; t <= Tx; ++t)
      for (int u = 0; u <= Ty; ++u) {
        int v = 0;
        for (; v < Tz; v += 2, e += 2) {
          acc0 = fma(Ep[e], Yh[hidx(t, u, v) * ncd + kc], acc0);
          acc1 = fma(Ep[e + 1], Yh[hidx(t, u, v + 1) * ncd + kc], acc1);
        }
        if (v == Tz) {
          acc0 = fma(Ep[e], Yh[hidx(t, u, v) * ncd + kc], acc0);
          ++e;
        }
      }
    eri[it] = acc0 + acc1;
  }
}

// One contracted quartet on a group of G lanes, in FP64 (Real = double) or
// in FP32 (Real = float, the mixed-precision path below the cutoff: FP32
// table, pair-relative centres, FP32 copies of U, E and D, exact FP32->FP64
// conversion of every digested element before the FP64 atomic add).
template <int G, class Real>
__device__ void quartet_body(const KArgs &a, const ClassTables &ct, double *scr_d, int P, int Q, int gl,
                             unsigned gmask, const MolView &mv) {
  constexpr bool F32 = sizeof(Real) == 4;
  const DevPairs &dp = a.dp;
  const int2 ab = dp.ab[P], cd = dp.ab[Q];
  const int sA = ab.x, sB = ab.y, sC = cd.x, sD = cd.y;
  const int cb = dp.cls[P], ck = dp.cls[Q];
  const int la = dp.sl[sA], lb = dp.sl[sB], lc = dp.sl[sC], ld = dp.sl[sD];
  const int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
  const int nab = na * nb, ncd = nc * nd;
  const int Lab = la + lb, Lcd = lc + ld, L = Lab + Lcd;
  const int nhab = nherm(Lab), nhL = nherm(L);
  FK_CHECK((F32 ? (nab * ncd + nhab * ncd + 2 * nhL + L + 2) / 2 : nab * ncd + nhab * ncd + 2 * nhL + L + 1) <=
               a.stride,
           1, a.stride);
  FK_CHECK(P >= 0 && P < dp.npair && Q >= 0 && Q < dp.npair, 2, Q);
  FK_CHECK(dp.prim[P].x >= 0 && dp.prim[P].x + dp.prim[P].y <= a.nprimtot, 3, dp.prim[P].x);
  FK_CHECK(dp.prim[Q].x >= 0 && dp.prim[Q].x + dp.prim[Q].y <= a.nprimtot, 4, dp.prim[Q].x);
  FK_CHECK(dp.eoff[dp.prim[P].x + dp.prim[P].y - 1] + ct.nE[cb] <= a.nEtot, 5, cb);
  FK_CHECK(dp.eoff[dp.prim[Q].x + dp.prim[Q].y - 1] + ct.nE[ck] <= a.nEtot, 6, ck);
  FK_CHECK(dp.sbf[sA] + na <= mv.N && dp.sbf[sB] + nb <= mv.N && dp.sbf[sC] + nc <= mv.N &&
               dp.sbf[sD] + nd <= mv.N, 7, sA);
  FK_CHECK(L <= LTOT && nab <= MAXCP && ncd <= MAXCP, 8, L);
  Real *scr = reinterpret_cast<Real *>(scr_d);
  Real *eri = scr;
  Real *Yh = eri + nab * ncd;
  Real *R0 = Yh + nhab * ncd;
  Real *R1 = R0 + nhL;
  Real *F = R1 + nhL;
  const Real *Epool;
  if constexpr (F32)
    Epool = dp.Ef;
  else
    Epool = dp.E;
  float ACx = 0.f, ACy = 0.f, ACz = 0.f;
  if constexpr (F32) {
    const float *ha = dp.shl + 6 * sA, *hc = dp.shl + 6 * sC;
    ACx = (ha[0] - hc[0]) + (ha[3] - hc[3]);
    ACy = (ha[1] - hc[1]) + (ha[4] - hc[4]);
    ACz = (ha[2] - hc[2]) + (ha[5] - hc[5]);
  }

  for (int i = gl; i < nab * ncd; i += G) eri[i] = Real(0);
  const int2 pb = dp.prim[P], pk = dp.prim[Q];
  // primitive-quartet screening; the decision is the same on every lane of
  // the group, so the group leaves its loops together
  const PrimScreen ps = prim_screen(a, mv, sA, sB, sC, sD);
  for (int ip = pb.x; ip < pb.x + pb.y; ++ip) {
    if (prim_skip(a, mv, ps, ip, pk.x)) break;
    const Real *EP = Epool + dp.eoff[ip];
    for (int i = gl; i < nhab * ncd; i += G) Yh[i] = Real(0);
    for (int jq = pk.x; jq < pk.x + pk.y; ++jq) {
      if (prim_skip(a, mv, ps, ip, jq)) break;
      const Real *EQ = Epool + dp.eoff[jq];
      Real X, Y, Z;
      if constexpr (F32) {
        const float4 PA = dp.paf[ip], QC = dp.paf[jq];
        X = PA.x - QC.x + ACx;
        Y = PA.y - QC.y + ACy;
        Z = PA.z - QC.z + ACz;
        const float rs = rsqrtf(PA.w + QC.w);
        const float alpha = (PA.w * QC.w) * (rs * rs);
        const float T = alpha * fmaf(X, X, fmaf(Y, Y, Z * Z));
        boys_seeds_rt_f32<G>(a.boysf, T, rs, -2.0f * alpha, L, F, R0, gl);
      } else {
        const PrimQuartet q = prim_quartet(dp.pz[ip], dp.pf[ip], dp.pz[jq], dp.pf[jq]);
        FK_CHECK(q.T >= 0.0 && q.T == q.T && q.gi <= BOYS_NGRID - 1, 9, jq);
        X = q.X;
        Y = q.Y;
        Z = q.Z;
        boys_seeds_rt<G>(a.boys, q, L, F, R0, gl, a.boysf);
      }
      group_sync(gmask, G);
      const Real *R = hermite_r<G, Real>(ct, L, X, Y, Z, F, R0, R1, gl, gmask);
      ket_transform<G, Real>(ct, EQ, R, Yh, nhab, ncd, nd, lc, ld, ck, gl);
      group_sync(gmask, G);
    }
    bra_transform<G, Real>(ct, EP, Yh, eri, nab, ncd, nb, la, lb, cb, gl);
    group_sync(gmask, G);
  }
  // digestion into J and K (Sec. 2.3 eight-fold symmetry; J = Jt + Jt^T and
  // K = Kt + Kt^T are formed afterwards by the symmetrisation kernel)
  Real fac = Real(1);
  if (sA == sB) fac *= Real(0.5);
  if (sC == sD) fac *= Real(0.5);
  if (P == Q) fac *= Real(0.5);
  const int N = mv.N;
  const int fa = dp.sbf[sA], fb = dp.sbf[sB], fc = dp.sbf[sC], fd = dp.sbf[sD];
  const Real *Dm;
  if constexpr (F32)
    Dm = mv.Df;
  else
    Dm = mv.D;
  const Real fac2 = Real(2) * fac;
  const int n1 = nab, n2 = n1 + ncd, n3 = n2 + na * nc, n4 = n3 + na * nd, n5 = n4 + nb * nc,
            n6 = n5 + nb * nd;
  // FP32 bodies and groups of up to 8 lanes stage the density sub-blocks;
  // the FP64 bodies of 16- and 32-lane groups read D in place, which
  // measured faster there (the staging round trip is not repaid by the
  // few outputs per lane).
  constexpr bool kStage = F32 || G <= 8;
  if constexpr (kStage) {
    // The six density sub-blocks D_ab, D_cd, D_ac, D_ad, D_bc, D_bd, each a
    // row-major block with row stride ldb: staged once in the scratch the
    // transforms no longer need (Yh, R0, R1, F) when they fit there, else read
    // from D in place (row stride N).
    const Real *Db[6];
    int ldb[6];
    const int r0[6] = {fa, fc, fa, fa, fb, fb}, c0[6] = {fb, fd, fc, fd, fc, fd};
    const int nr[6] = {na, nc, na, na, nb, nb}, ncl[6] = {nb, nd, nc, nd, nc, nd};
    const int nstage = nab + ncd + (na + nb) * (nc + nd);
    if (nstage <= nhab * ncd + 2 * nhL + L + 1) {
      Real *Ds = Yh;
      int off = 0;
      for (int k = 0; k < 6; ++k) {
        Db[k] = Ds + off;
        ldb[k] = ncl[k];
        const int nk = nr[k] * ncl[k];
        for (int i = gl; i < nk; i += G) {
          const int r = i / ncl[k], c = i - r * ncl[k];
          Ds[off + i] = Dm[(size_t)(r0[k] + r) * N + c0[k] + c];
        }
        off += nk;
      }
      group_sync(gmask, G);
    } else {
      for (int k = 0; k < 6; ++k) {
        Db[k] = Dm + (size_t)r0[k] * N + c0[k];
        ldb[k] = N;
      }
    }
    // sum_{i < no, j < ni} x[i so + j si] y[i ldy + j] over two independent
    // chains (even / odd j)
    auto dot2d = [](const Real *x, int so, int si, const Real *y, int ldy, int no, int ni) -> Real {
      Real s0 = Real(0), s1 = Real(0);
      for (int i = 0; i < no; ++i, x += so, y += ldy) {
        int j = 0;
        for (; j + 1 < ni; j += 2) {
          s0 = fma(x[j * si], y[j], s0);
          s1 = fma(x[(j + 1) * si], y[j + 1], s1);
        }
        if (j < ni) s0 = fma(x[j * si], y[j], s0);
      }
      return s0 + s1;
    };
    // J outputs are o < n2, K outputs n2 <= o < n6: only the built parts
    const int o0 = (a.parts & 1) ? 0 : n2, o1 = (a.parts & 2) ? n6 : n2;
    const int scd = ncd, sbcd = nb * ncd;  // eri strides of the b and a indices
    for (int o = o0 + gl; o < o1; o += G) {
      Real s;
      double *dst;
      if (o < n1) {  // J_ab += (ab|cd) D_cd
        const int ia = o / nb, ib = o - ia * nb;
        s = fac2 * dot2d(eri + (size_t)o * ncd, nd, 1, Db[1], ldb[1], nc, nd);
        dst = mv.J + (size_t)(fa + ia) * N + fb + ib;
      } else if (o < n2) {  // J_cd += (ab|cd) D_ab
        const int k = o - n1, ic = k / nd, id = k - ic * nd;
        s = fac2 * dot2d(eri + k, sbcd, scd, Db[0], ldb[0], na, nb);
        dst = mv.J + (size_t)(fc + ic) * N + fd + id;
      } else if (o < n3) {  // K_ac += (ab|cd) D_bd
        const int k = o - n2, ia = k / nc, ic = k - ia * nc;
        s = fac * dot2d(eri + (size_t)ia * sbcd + ic * nd, scd, 1, Db[5], ldb[5], nb, nd);
        dst = mv.K + (size_t)(fa + ia) * N + fc + ic;
      } else if (o < n4) {  // K_ad += (ab|cd) D_bc
        const int k = o - n3, ia = k / nd, id = k - ia * nd;
        s = fac * dot2d(eri + (size_t)ia * sbcd + id, scd, nd, Db[4], ldb[4], nb, nc);
        dst = mv.K + (size_t)(fa + ia) * N + fd + id;
      } else if (o < n5) {  // K_bc += (ab|cd) D_ad
        const int k = o - n4, ib = k / nc, ic = k - ib * nc;
        s = fac * dot2d(eri + (size_t)ib * scd + ic * nd, sbcd, 1, Db[3], ldb[3], na, nd);
        dst = mv.K + (size_t)(fb + ib) * N + fc + ic;
      } else {  // K_bd += (ab|cd) D_ac
        const int k = o - n5, ib = k / nd, id = k - ib * nd;
        s = fac * dot2d(eri + (size_t)ib * scd + id, sbcd, nd, Db[2], ldb[2], na, nc);
        dst = mv.K + (size_t)(fb + ib) * N + fd + id;
      }
      if constexpr (F32)
        atomicAdd(dst, f2d_any(s));
      else
        atomicAdd(dst, s);
    }
  } else {
    // sum_m x(m) y(m) over two independent chains (even / odd m)
    auto dot2 = [](int n, auto &&xy) -> Real {
      Real s0 = Real(0), s1 = Real(0), x, y;
      int m = 0;
      for (; m + 1 < n; m += 2) {
        xy(m, x, y);
        s0 = fma(x, y, s0);
        xy(m + 1, x, y);
        s1 = fma(x, y, s1);
      }
      if (m < n) {
        xy(m, x, y);
        s0 = fma(x, y, s0);
      }
      return s0 + s1;
    };
    // J outputs are o < n2, K outputs n2 <= o < n6: only the built parts
    const int o0 = (a.parts & 1) ? 0 : n2, o1 = (a.parts & 2) ? n6 : n2;
    for (int o = o0 + gl; o < o1; o += G) {
      Real s;
      double *dst;
      if (o < n1) {  // J_ab += (ab|cd) D_cd
        const int ia = o / nb, ib = o - ia * nb;
        const Real *e = eri + (size_t)o * ncd;
        s = dot2(ncd, [&](int m, Real &x, Real &y) {
          const int ic = m / nd, id = m - ic * nd;
          x = e[m];
          y = Dm[(size_t)(fc + ic) * N + fd + id];
        });
        dst = mv.J + (size_t)(fa + ia) * N + fb + ib;
        s *= fac2;
      } else if (o < n2) {  // J_cd += (ab|cd) D_ab
        const int k = o - n1, ic = k / nd, id = k - ic * nd;
        s = dot2(nab, [&](int m, Real &x, Real &y) {
          const int ia = m / nb, ib = m - ia * nb;
          x = eri[(size_t)m * ncd + k];
          y = Dm[(size_t)(fa + ia) * N + fb + ib];
        });
        dst = mv.J + (size_t)(fc + ic) * N + fd + id;
        s *= fac2;
      } else if (o < n3) {  // K_ac += (ab|cd) D_bd
        const int k = o - n2, ia = k / nc, ic = k - ia * nc;
        s = dot2(nb * nd, [&](int m, Real &x, Real &y) {
          const int ib = m / nd, id = m - ib * nd;
          x = eri[((ia * nb + ib) * nc + ic) * nd + id];
          y = Dm[(size_t)(fb + ib) * N + fd + id];
        });
        dst = mv.K + (size_t)(fa + ia) * N + fc + ic;
        s *= fac;
      } else if (o < n4) {  // K_ad += (ab|cd) D_bc
        const int k = o - n3, ia = k / nd, id = k - ia * nd;
        s = dot2(nb * nc, [&](int m, Real &x, Real &y) {
          const int ib = m / nc, ic = m - ib * nc;
          x = eri[((ia * nb + ib) * nc + ic) * nd + id];
          y = Dm[(size_t)(fb + ib) * N + fc + ic];
        });
        dst = mv.K + (size_t)(fa + ia) * N + fd + id;
        s *= fac;
      } else if (o < n5) {  // K_bc += (ab|cd) D_ad
        const int k = o - n4, ib = k / nc, ic = k - ib * nc;
        s = dot2(na * nd, [&](int m, Real &x, Real &y) {
          const int ia = m / nd, id = m - ia * nd;
          x = eri[((ia * nb + ib) * nc + ic) * nd + id];
          y = Dm[(size_t)(fa + ia) * N + fd + id];
        });
        dst = mv.K + (size_t)(fb + ib) * N + fc + ic;
        s *= fac;
      } else {  // K_bd += (ab|cd) D_ac
        const int k = o - n5, ib = k / nd, id = k - ib * nd;
        s = dot2(na * nc, [&](int m, Real &x, Real &y) {
          const int ia = m / nc, ic = m - ia * nc;
          x = eri[((ia * nb + ib) * nc + ic) * nd + id];
          y = Dm[(size_t)(fa + ia) * N + fc + ic];
        });
        dst = mv.K + (size_t)(fb + ib) * N + fd + id;
        s *= fac;
      }
      if constexpr (F32)
        atomicAdd(dst, f2d_any(s));
      else
        atomicAdd(dst, s);
    }
  }
  group_sync(gmask, G);
}

// MODE 0: every surviving quartet in FP64 (FP64 build).  Mixed build, one
// launch per part: MODE 1 takes the survivors whose bound is at least the FP32
// cutoff (FP64 body), MODE 2 those below it (FP32 body).  Each launch holds a
// single body, so a warp never alternates between the two.
// The FP32 part (MODE 2) keeps its intermediates in half the shared memory of
// the FP64 body, so more of its blocks fit on an SM; its register budget is
// capped to match (five blocks of four warps; the FP64 bodies keep the
// budget of four blocks, 128 registers).
template <int G, int MODE>
__global__ void __launch_bounds__(128, MODE == 2 ? 5 : 4) k_jk(KArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {
    const int *src = reinterpret_cast<const int *>(a.tabs);
    int *dst = reinterpret_cast<int *>(smem_raw);
    for (int i = threadIdx.x; i < (int)(sizeof(ClassTables) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const ClassTables &ct = *reinterpret_cast<const ClassTables *>(smem_raw);
  double *scr_base = reinterpret_cast<double *>(smem_raw + TAB_BYTES);
  constexpr int NG = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane - grp * G;
  double *scr = scr_base + (size_t)(warp * NG + grp) * a.stride;
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
  // Warp-level work queue, as in the register kernels: the unit's kets are
  // screened 32 at a time and the survivors of this launch's part appended to
  // a queue that is drained NG quartets at a time (one per group), so no
  // group holds a screened quartet while the others compute.
  __shared__ int queues[4][64];
  int *q64 = queues[warp];
  const unsigned lt = (1u << lane) - 1u;
  auto drain = [&](int *q, int &n, const MolView &mv, int P, bool all) {
    const int k = all ? n : (n / NG) * NG;
    for (int i = 0; i < k; i += NG)
      if (i + grp < k) {
        if constexpr (MODE == 2)
          quartet_body<G, float>(a, ct, scr, P, q[i + grp], gl, gmask, mv);
        else
          quartet_body<G, double>(a, ct, scr, P, q[i + grp], gl, gmask, mv);
      }
    __syncwarp();
    const int rest = n - k;  // < NG <= 32 entries move to the front
    const int v = lane < rest ? q[k + lane] : 0;
    __syncwarp();
    if (lane < rest) q[lane] = v;
    n = rest;
    __syncwarp();
  };
  for (;;) {
    const int u = next_unit(a.counter, lane);
    if (u >= a.nunits) break;
    const Unit un = a.units[u];
    const int P = un.bra;
    const int2 ab = a.dp.ab[P];
    const MolView mv = mol_view(a, ab.x);
    int n64 = 0;
    for (int c = un.k0; c < un.k1; c += 32) {
      const int Q = c + lane;
      float b = -1.0f;
      if (Q < un.k1) {
        const int2 cd = a.dp.ab[Q];
        b = quartet_bound(a, mv, ab.x, ab.y, cd.x, cd.y, P, Q);
      }
      bool keep = b >= 0.0f;
      if constexpr (MODE == 1) keep = keep && !(b < a.fp32_cutoff_f);
      if constexpr (MODE == 2) keep = keep && b < a.fp32_cutoff_f;
      const unsigned m64 = __ballot_sync(0xffffffffu, keep);
      if (keep) q64[n64 + __popc(m64 & lt)] = Q;
      n64 += __popc(m64);
      __syncwarp();
      if (n64 >= NG) drain(q64, n64, mv, P, false);
    }
    if (n64 > 0) drain(q64, n64, mv, P, true);
  }
}

// Schwarz factors from diagonal integrals (Eqs. cauchy-schwarz 1, 2): one
// warp per contracted pair; lanes own Cartesian pairs kc; for every primitive
// quartet [ij|ij] ... all (i,j): the diagonal (kc|kc) element is
// sum_p E^i_p sum_q (-1)^{|q|} E^j_q R_{p+q}.
__global__ void __launch_bounds__(128) k_schwarz(DevPairs dp, const double *boys, const ClassTables *tabs,
                                                 double *Gpair, double *Gprim) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {
    const int *src = reinterpret_cast<const int *>(tabs);
    int *dst = reinterpret_cast<int *>(smem_raw);
    for (int i = threadIdx.x; i < (int)(sizeof(ClassTables) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const ClassTables &ct = *reinterpret_cast<const ClassTables *>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *scr = reinterpret_cast<double *>(smem_raw + TAB_BYTES) + warp * (2 * NHMAX + LTOT + 2);
  double *R0 = scr, *R1 = scr + NHMAX, *F = scr + 2 * NHMAX;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int P = blockIdx.x * (blockDim.x >> 5) + warp; P < dp.npair; P += nw) {
    const int2 ab = dp.ab[P];
    const int la = dp.sl[ab.x], lb = dp.sl[ab.y], c = dp.cls[P];
    const int nb = ncart(lb), nab = ncart(la) * nb, L = 2 * (la + lb);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int2 pr = dp.prim[P];
    for (int i = pr.x; i < pr.x + pr.y; ++i) {
      const PZ P4 = dp.pz[i];
      const float4 Pf = dp.pf[i];
      for (int j = pr.x; j < pr.x + pr.y; ++j) {
        const PrimQuartet q = prim_quartet(P4, Pf, dp.pz[j], dp.pf[j]);
        boys_seeds_rt<32>(boys, q, L, F, R0, lane);
        __syncwarp();
        const double *R = hermite_r<32>(ct, L, q.X, q.Y, q.Z, F, R0, R1, lane, 0xffffffffu);
        double pm = 0.0;
        for (int r = 0; r < 4; ++r) {
          const int kc = lane + 32 * r;
          if (kc >= nab) break;
          const int ia = kc / nb, ib = kc - ia * nb;
          const uint8_t *ac = ct.comp[la][ia], *bc = ct.comp[lb][ib];
          const int Tx = ac[0] + bc[0], Ty = ac[1] + bc[1], Tz = ac[2] + bc[2];
          const double *Ei = dp.E + dp.eoff[i] + ct.eoff[c][kc];
          const double *Ej = dp.E + dp.eoff[j] + ct.eoff[c][kc];
          double v = 0.0;
          int e1 = 0;
          for (int t1 = 0; t1 <= Tx; ++t1)
            for (int u1 = 0; u1 <= Ty; ++u1)
              for (int v1 = 0; v1 <= Tz; ++v1, ++e1) {
                double inner = 0.0;
                int e2 = 0;
                for (int t2 = 0; t2 <= Tx; ++t2)
                  for (int u2 = 0; u2 <= Ty; ++u2)
                    for (int v2 = 0; v2 <= Tz; ++v2, ++e2) {
                      const double rr = R[hidx(t1 + t2, u1 + u2, v1 + v2)];
                      inner = ((t2 + u2 + v2) & 1) ? fma(-Ej[e2], rr, inner) : fma(Ej[e2], rr, inner);
                    }
                v = fma(Ei[e1], inner, v);
              }
          acc[r] += v;
          pm = fmax(pm, fabs(v));
        }
        if (i == j) {
          for (int o = 16; o > 0; o >>= 1) pm = fmax(pm, __shfl_xor_sync(0xffffffffu, pm, o));
          if (lane == 0) Gprim[i] = sqrt(pm);
        }
        __syncwarp();
      }
    }
    double mx = 0.0;
    for (int r = 0; r < 4; ++r)
      if (lane + 32 * r < nab) mx = fmax(mx, acc[r]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) Gpair[P] = sqrt(fmax(mx, 0.0));
  }
}

// Shell-block maxima |D| (Sec. 3.2 density screening) and a finiteness check.
__global__ void k_dprep(const double *__restrict__ D, int N, const int *__restrict__ sbf,
                        const int *__restrict__ sl, int ns, double *__restrict__ Dsh, float *__restrict__ Df,
                        float *__restrict__ Dshf) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ns * ns) return;
  const int a = idx / ns, b = idx - a * ns;
  const int fa = sbf[a], fb = sbf[b], na = ncart(sl[a]), nb = ncart(sl[b]);
  double mx = 0.0;
  bool bad = false;
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j) {
      const double v = D[(size_t)(fa + i) * N + fb + j];
      if (Df) Df[(size_t)(fa + i) * N + fb + j] = (float)v;
      if (!isfinite(v)) bad = true;
      mx = fmax(mx, fabs(v));
    }
  if (bad) atomicCAS(&g_status, 0, (int)FOCK_ERR_NONFINITE);
  Dsh[idx] = bad ? INFINITY : mx;
  if (Dshf) Dshf[idx] = bad ? INFINITY : (float)mx;
}

// --------------------------------------------------------------------------
// Decay bound of the density (Sec. 4.3.1, Eq. density_bound)
// --------------------------------------------------------------------------
// Centre distance of shells a and b, rounded the same way as a plain
// left-to-right evaluation (no fused multiply-adds), so that the 0.5-bohr bin
// of a pair is reproducible by any IEEE implementation.
__device__ __forceinline__ double centre_distance(const double *xyz, int a, int b) {
  const double dx = __dsub_rn(xyz[3 * a], xyz[3 * b]);
  const double dy = __dsub_rn(xyz[3 * a + 1], xyz[3 * b + 1]);
  const double dz = __dsub_rn(xyz[3 * a + 2], xyz[3 * b + 2]);
  return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

constexpr double DECAY_BIN = 0.5;  // bohr

// Largest shell-block maximum of |D| per distance bin, over pairs of shells on
// different atoms (same-atom elements would skew the decay, Sec. 4.3.1).
// Non-negative doubles order like their bit patterns, so the maximum is an
// integer atomicMax.
__global__ void k_decay_bins(DevPairs dp, const double *__restrict__ Dsh, int nbins,
                             unsigned long long *__restrict__ bins) {
  const int ns = dp.nshell;
  const long long n = (long long)ns * ns;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(idx / ns), b = (int)(idx - (long long)a * ns);
    if (b <= a || dp.satom[a] == dp.satom[b]) continue;
    const double v = Dsh[idx];
    if (!(v > 0.0) || !isfinite(v)) continue;
    int k = (int)floor(centre_distance(dp.sxyz, a, b) / DECAY_BIN);
    if (k >= nbins) k = nbins - 1;
    atomicMax(bins + k, (unsigned long long)__double_as_longlong(v));
  }
}

// Least-squares line ln max|D| = ln H - Lambda r through the non-empty bins
// (r the bin centre), then ln H raised so that the line lies above each bin's
// maximum over the whole bin (its far edge when Lambda > 0).  Fewer than two
// bins: Lambda = 0, H the largest maximum.  One block.
__global__ void k_decay_fit(const unsigned long long *__restrict__ bins, int nbins, double *__restrict__ HL) {
  __shared__ double red[5][256];
  double n = 0, sx = 0, sy = 0, sxx = 0, sxy = 0;
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
    const double v = __longlong_as_double((long long)bins[i]);
    if (!(v > 0.0)) continue;
    const double x = (i + 0.5) * DECAY_BIN, y = log(v);
    n += 1;
    sx += x;
    sy += y;
    sxx += x * x;
    sxy += x * y;
  }
  red[0][threadIdx.x] = n;
  red[1][threadIdx.x] = sx;
  red[2][threadIdx.x] = sy;
  red[3][threadIdx.x] = sxx;
  red[4][threadIdx.x] = sxy;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 5; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  n = red[0][0];
  sx = red[1][0];
  sy = red[2][0];
  sxx = red[3][0];
  sxy = red[4][0];
  double lam = 0.0;
  if (n >= 2.0) {
    const double den = n * sxx - sx * sx;
    if (den > 0.0) lam = -(n * sxy - sx * sy) / den;
  }
  __syncthreads();
  // ln H = max over bins of y + Lambda * edge
  double m = -INFINITY;
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
    const double v = __longlong_as_double((long long)bins[i]);
    if (!(v > 0.0)) continue;
    const double edge = (lam > 0.0 ? i + 1 : i) * DECAY_BIN;
    m = fmax(m, log(v) + lam * edge);
  }
  red[0][threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    HL[0] = red[0][0] == -INFINITY ? 0.0 : exp(red[0][0]);
    HL[1] = lam;
  }
}

// C = A B (transB = 0) or A B^T (transB = 1) for n x n row-major FP32
// matrices: 32 x 32 output tiles, 16 x 16 threads with 2 x 2 outputs each,
// K steps of 32 staged in shared memory; ragged edges read as zero.
__global__ void k_sgemm_nn(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C, int n,
                           int transB) {
  __shared__ float As[32][33], Bs[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int i = ty; i < 32; i += 16)
      for (int j = tx; j < 32; j += 16) {
        const int r = r0 + i, k = k0 + j;
        As[i][j] = (r < n && k < n) ? A[(size_t)r * n + k] : 0.f;
        const int kb = k0 + i, c = c0 + j;
        Bs[i][j] = (kb < n && c < n) ? (transB ? B[(size_t)c * n + kb] : B[(size_t)kb * n + c]) : 0.f;
      }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float a0 = As[ty][k], a1 = As[ty + 16][k], b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
      if (r < n && c < n) C[(size_t)r * n + c] = acc[i][j];
    }
}

// W_xy = H exp(-Lambda (|XY| - R_x - R_y)): for every kept pair (x z) and
// (y w), |ZW| >= |XY| - R_x - R_y, so W_xy bounds |D_zw|.  Where that distance
// bound is not positive the partners may share an atom (elements the fit
// excludes) and no bound is used (+inf).
// With GDG (the block bound (A Dsh A^T)_xy >= max |K_xy|, A_xz = n_z G_xz
// over kept pairs, Sec. 4.3.1's comparison with Luehr et al.) below tau*, the
// whole block K_xy is negligible and W_xy = 0 drops its contributions.
__global__ void k_decay_w(DevPairs dp, const double *__restrict__ HL, const float *__restrict__ GDG, float kthr,
                          float *__restrict__ W) {
  const int ns = dp.nshell;
  const long long n = (long long)ns * ns;
  const double H = HL[0], lam = HL[1];
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(idx / ns), y = (int)(idx - (long long)x * ns);
    const double r = centre_distance(dp.sxyz, x, y) - (double)dp.sRG[x].x - (double)dp.sRG[y].x;
    float w = r > 0.0 ? (float)(H * exp(-lam * r)) : INFINITY;
    // FP32 sums of non-negative terms: a relative margin of 1e-4 covers
    // their rounding, so the test only drops blocks the exact bound drops
    if (GDG && fmaxf(GDG[idx], GDG[(long long)y * ns + x]) * 1.0001f < kthr) w = 0.0f;
    W[idx] = w;
  }
}

cudaError_t launch_decay_bound(const DevPairs &dp, const double *Dsh, int nbins, double *bins, double *HL, float *W,
                               cudaStream_t st, const float *Gn, const float *Dshf, float *T, float *GDG,
                               double k_thresh) {
  if (nbins < 1 || !dp.satom || !dp.sRG) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(double) * nbins, st);
  if (e != cudaSuccess) return e;
  const long long n = (long long)dp.nshell * dp.nshell;
  const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 16);
  k_decay_bins<<<grid, 256, 0, st>>>(dp, Dsh, nbins, reinterpret_cast<unsigned long long *>(bins));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_decay_fit<<<1, 256, 0, st>>>(reinterpret_cast<const unsigned long long *>(bins), nbins, HL);
  e = cudaGetLastError();
  if (e != cudaSuccess || !W) return e;
  const bool gdg = Gn && Dshf && T && GDG;
  if (gdg) {
    const int ns = dp.nshell;
    dim3 blk(16, 16), grd((ns + 31) / 32, (ns + 31) / 32);
    k_sgemm_nn<<<grd, blk, 0, st>>>(Gn, Dshf, T, ns, 0);    // T = A Dsh
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sgemm_nn<<<grd, blk, 0, st>>>(T, Gn, GDG, ns, 1);     // GDG = T A^T
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_decay_w<<<grid, 256, 0, st>>>(dp, HL, gdg ? GDG : nullptr, (float)k_thresh, W);
  return cudaGetLastError();
}

// M <- M + M^T in place, for J (z = 0) and K (z = 1).
__global__ void k_symmetrize(double *J, double *K, int n) {
  double *M = (blockIdx.z == 0 && J) ? J : K;  // J or K may be absent (one z slice)
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n || i > j) return;
  if (i == j) {
    M[(size_t)i * n + i] *= 2.0;
  } else {
    const double s = M[(size_t)i * n + j] + M[(size_t)j * n + i];
    M[(size_t)i * n + j] = s;
    M[(size_t)j * n + i] = s;
  }
}

// --------------------------------------------------------------------------
// batched builds: one launch over every molecule (packed index spaces)
// --------------------------------------------------------------------------
__device__ __forceinline__ int find_mol(const long long *prefix, int nmol, long long idx) {
  int lo = 0, hi = nmol;  // prefix[lo] <= idx < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= idx)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__global__ void k_zero_batch(const MolEntry *__restrict__ mt, const long long *__restrict__ n2p, int nmol,
                             long long total) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m = find_mol(n2p, nmol, idx);
    const long long r = idx - n2p[m];
    mt[m].J[r] = 0.0;
    mt[m].K[r] = 0.0;
  }
}

__global__ void k_dprep_batch(const MolEntry *__restrict__ mt, const long long *__restrict__ dshp, int nmol,
                              long long total, const int *__restrict__ sbf, const int *__restrict__ sl,
                              double *__restrict__ Dsh, float *__restrict__ Dshf) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m = find_mol(dshp, nmol, idx);
    const MolEntry &e = mt[m];
    const int r = (int)(idx - dshp[m]);
    const int a = e.s0 + r / e.ns, b = e.s0 + r % e.ns;
    const int fa = sbf[a], fb = sbf[b], na = ncart(sl[a]), nb = ncart(sl[b]);
    double mx = 0.0;
    bool bad = false;
    for (int i = 0; i < na; ++i)
      for (int j = 0; j < nb; ++j) {
        const size_t o = (size_t)(fa + i) * e.N + fb + j;
        const double v = e.D[o];
        if (e.Df) const_cast<float *>(e.Df)[o] = (float)v;
        if (!isfinite(v)) bad = true;
        mx = fmax(mx, fabs(v));
      }
    if (bad) atomicCAS(&g_status, 0, (int)FOCK_ERR_NONFINITE);
    Dsh[idx] = bad ? INFINITY : mx;
    Dshf[idx] = bad ? INFINITY : (float)mx;
  }
}

__global__ void k_symmetrize_batch(const MolEntry *__restrict__ mt, const long long *__restrict__ n2p, int nmol,
                                   long long total) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m = find_mol(n2p, nmol, idx);
    const MolEntry &e = mt[m];
    const int r = (int)(idx - n2p[m]);
    const int i = r / e.N, j = r % e.N;
    if (i > j) continue;
    for (int z = 0; z < 2; ++z) {
      double *M = z == 0 ? e.J : e.K;
      if (i == j) {
        M[(size_t)i * e.N + i] *= 2.0;
      } else {
        const double s = M[(size_t)i * e.N + j] + M[(size_t)j * e.N + i];
        M[(size_t)i * e.N + j] = s;
        M[(size_t)j * e.N + i] = s;
      }
    }
  }
}

static int grid_for(long long total) {
  long long b = (total + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b > 0 ? b : 1);
}

cudaError_t launch_zero_batch(const MolEntry *mt, const long long *n2p, int nmol, long long total, cudaStream_t st) {
  k_zero_batch<<<grid_for(total), 256, 0, st>>>(mt, n2p, nmol, total);
  return cudaGetLastError();
}
cudaError_t launch_dprep_batch(const MolEntry *mt, const long long *dshp, int nmol, long long total, const int *sbf,
                               const int *sl, double *Dsh, float *Dshf, cudaStream_t st) {
  k_dprep_batch<<<grid_for(total), 256, 0, st>>>(mt, dshp, nmol, total, sbf, sl, Dsh, Dshf);
  return cudaGetLastError();
}
cudaError_t launch_symmetrize_batch(const MolEntry *mt, const long long *n2p, int nmol, long long total,
                                    cudaStream_t st) {
  k_symmetrize_batch<<<grid_for(total), 256, 0, st>>>(mt, n2p, nmol, total);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// host-side launch helpers
// --------------------------------------------------------------------------

cudaError_t upload_tables(cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (s_boys[dev] && s_tabs[dev] && s_boysf[dev]) return cudaSuccess;
  const std::vector<double> &bt = boys_table();
  std::vector<float> btf(bt.begin(), bt.end());
  double *b = nullptr;
  float *bf = nullptr;
  ClassTables *t = nullptr;
  if ((e = cudaMalloc(&b, bt.size() * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&bf, btf.size() * sizeof(float))) != cudaSuccess) {
    cudaFree(b);
    return e;
  }
  if ((e = cudaMalloc(&t, sizeof(ClassTables))) != cudaSuccess) {
    cudaFree(b);
    cudaFree(bf);
    return e;
  }
  e = cudaMemcpyAsync(b, bt.data(), bt.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bf, btf.data(), btf.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t, &class_tables(), sizeof(ClassTables), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(b);
    cudaFree(bf);
    cudaFree(t);
    return e;
  }
  s_boys[dev] = b;
  s_boysf[dev] = bf;
  s_tabs[dev] = t;
  return cudaSuccess;
}

const double *dev_boys() {
  int dev = 0;
  cudaGetDevice(&dev);
  return s_boys[dev];
}
const float *dev_boys_f() {
  int dev = 0;
  cudaGetDevice(&dev);
  return s_boysf[dev];
}
const ClassTables *dev_class_tables() {
  int dev = 0;
  cudaGetDevice(&dev);
  return s_tabs[dev];
}

cudaError_t launch_schwarz(const DevPairs &dp, double *Gpair, double *Gprim, cudaStream_t st) {
  if (dp.npair == 0) return cudaSuccess;
  const size_t smem = TAB_BYTES + 4 * (2 * NHMAX + LTOT + 2) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_schwarz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int blocks = (dp.npair + 3) / 4;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_schwarz<<<blocks, 128, smem, st>>>(dp, dev_boys(), dev_class_tables(), Gpair, Gprim);
  return cudaGetLastError();
}

cudaError_t launch_dprep(const double *D, int nbf, const int *sbf, const int *sl, int nshell, double *Dsh,
                         cudaStream_t st, float *Df, float *Dshf) {
  const int n = nshell * nshell;
  k_dprep<<<(n + 255) / 256, 256, 0, st>>>(D, nbf, sbf, sl, nshell, Dsh, Df, Dshf);
  return cudaGetLastError();
}

cudaError_t launch_symmetrize(double *J, double *K, int n, cudaStream_t st) {
  const int nz = (J ? 1 : 0) + (K ? 1 : 0);
  if (nz == 0) return cudaSuccess;
  dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8, nz);
  k_symmetrize<<<grd, blk, 0, st>>>(J, K, n);
  return cudaGetLastError();
}

// The dynamic shared-memory limit of the group kernels is raised, never
// lowered (per device, to the largest size any tier has asked for): a CUDA
// graph's kernel nodes keep the sizes of the tiers they were captured from,
// and a node launched on its own (as a profiler replaying a graph node by node
// does) is checked against the function's current limit.  The call is repeated
// every time, so a limit lost with the context (cudaDeviceReset) comes back.
template <int G>
static cudaError_t set_smem_g(size_t smem) {
  static std::mutex mu;
  static int raised[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tracked = dev >= 0 && dev < 64;
  std::lock_guard<std::mutex> lock(mu);
  const int target = std::max((int)smem, tracked ? raised[dev] : 0);
  e = cudaFuncSetAttribute(k_jk<G, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, target);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_jk<G, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, target);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_jk<G, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, target);
  if (e == cudaSuccess && tracked) raised[dev] = target;
  return e;
}

// One group tier: a single FP64 launch, or in mixed mode (a.fp32_cutoff > 0)
// the FP64 part and then the FP32 part, each drawing units from its own counter.
template <int G>
static cudaError_t launch_g(const Tier &t, KArgs a, int threads, cudaStream_t st, int *counter2) {
  if (a.fp32_cutoff > 0.0) {
    if (!counter2) return cudaErrorInvalidValue;
    k_jk<G, 1><<<t.blocks, threads, t.smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    a.counter = counter2;
    if (t.r32_cb >= 0) return launch_reg32(t.r32_cb, t.r32_ck, a, t.blocks32, 128, st);
    a.stride = fp32_stride(t.stride);  // scratch counted in doubles, half of them needed
    k_jk<G, 2><<<t.blocks32 > 0 ? t.blocks32 : t.blocks, threads, t.smem32 > 0 ? t.smem32 : t.smem, st>>>(a);
  } else {
    k_jk<G, 0><<<t.blocks, threads, t.smem, st>>>(a);
  }
  return cudaGetLastError();
}

static cudaError_t launch_group(const Tier &t, const KArgs &a, int threads, cudaStream_t st, int *counter2) {
  switch (t.G) {
    case 1: return launch_g<1>(t, a, threads, st, counter2);
    case 2: return launch_g<2>(t, a, threads, st, counter2);
    case 4: return launch_g<4>(t, a, threads, st, counter2);
    case 8: return launch_g<8>(t, a, threads, st, counter2);
    case 16: return launch_g<16>(t, a, threads, st, counter2);
    case 32: return launch_g<32>(t, a, threads, st, counter2);
  }
  return cudaErrorInvalidValue;
}

template <int G>
static cudaError_t configure_g(Tier &t) {
  const size_t per_warp = (size_t)(32 / G) * t.stride * sizeof(double);
  const size_t per_warp32 = (size_t)(32 / G) * fp32_stride(t.stride) * sizeof(double);
  // 227 KB per block, less the kernel's static work queues
  const size_t limit = 227 * 1024 - sizeof(int) * 4 * 64;
  int wpb = 4;
  while (wpb > 1 && TAB_BYTES + wpb * per_warp > limit) --wpb;
  if (TAB_BYTES + wpb * per_warp > limit) return cudaErrorInvalidValue;
  t.warps_per_block = wpb;
  t.smem = TAB_BYTES + wpb * per_warp;
  cudaError_t e = set_smem_g<G>(t.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jk<G, 0>, 32 * wpb, t.smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm < 1) per_sm = 1;
  t.blocks = nsm * per_sm;
  const int need = (t.nunits + wpb - 1) / wpb;
  if (t.blocks > need) t.blocks = need > 0 ? need : 1;
  // FP32 part of a mixed tier: same warps per block, half the scratch; or
  // the class pair's FP32 register kernel (four warps per block)
  int per_sm32 = 0;
  int need32 = need;
  if (t.r32_cb >= 0) {
    t.smem32 = 0;
    e = occupancy_reg32(t.r32_cb, t.r32_ck, 128, &per_sm32);
    need32 = (t.nunits + 3) / 4;
  } else {
    t.smem32 = TAB_BYTES + wpb * per_warp32;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm32, k_jk<G, 2>, 32 * wpb, t.smem32);
  }
  if (e != cudaSuccess) return e;
  if (per_sm32 < 1) per_sm32 = 1;
  t.blocks32 = nsm * per_sm32;
  if (t.blocks32 > need32) t.blocks32 = need32 > 0 ? need32 : 1;
  return cudaSuccess;
}

cudaError_t configure_tier(Tier &t) {
  if (t.reg_cb >= 0) {
    t.warps_per_block = 4;
    t.smem = 0;
    int per_sm = 0;
    cudaError_t e = occupancy_reg(t.reg_cb, t.reg_ck, 128, t.mixed != 0, &per_sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm < 1) per_sm = 1;
    t.blocks = nsm * per_sm;
    const int need = (t.nunits + 3) / 4;
    if (t.blocks > need) t.blocks = need > 0 ? need : 1;
    return cudaSuccess;
  }
  switch (t.G) {
    case 1: return configure_g<1>(t);
    case 2: return configure_g<2>(t);
    case 4: return configure_g<4>(t);
    case 8: return configure_g<8>(t);
    case 16: return configure_g<16>(t);
    case 32: return configure_g<32>(t);
  }
  return cudaErrorInvalidValue;
}

// The dynamic shared-memory limit is a per-function attribute shared by
// every handle; make sure it covers this tier's need before launching.
static cudaError_t set_group_smem(const Tier &t) {
  switch (t.G) {
    case 1: return set_smem_g<1>(t.smem);
    case 2: return set_smem_g<2>(t.smem);
    case 4: return set_smem_g<4>(t.smem);
    case 8: return set_smem_g<8>(t.smem);
    case 16: return set_smem_g<16>(t.smem);
    case 32: return set_smem_g<32>(t.smem);
  }
  return cudaErrorInvalidValue;
}

static void set_screen_args(KArgs &a, double tau, const float *Dshf, double prim_eps,
                            const CallParts &cp = CallParts()) {
  a.parts = cp.parts;
  a.Wsh = cp.Wsh;
  a.k_thresh_f = (float)cp.k_thresh;
  a.Dshf = Dshf;
  a.tau_lo = (float)(tau * (1.0 - 1e-4));
  a.tau_hi = (float)(tau * (1.0 + 1e-4));
  a.tau_eps = prim_eps > 0.0 ? tau * prim_eps : 0.0;
  a.tau_eps_f = (float)a.tau_eps;
}

cudaError_t launch_jk_tier(const Tier &t, const DevPairs &dp, const double *D, const double *Dsh, double tau,
                           double prim_eps, double *J, double *K, int *counter, int *counter2, cudaStream_t st,
                           const float *Df, double fp32_cutoff, const float *Dshf, const CallParts &cp) {
  if (t.nunits == 0) return cudaSuccess;
  if (t.reg_cb >= 0) {
    KArgs a;
    a.dp = dp;
    a.nprimtot = dp.nprim_total;
    a.nEtot = dp.nE_total;
    a.D = D;
    a.Dsh = Dsh;
    a.tau = tau;
    a.J = J;
    a.K = K;
    a.units = t.d_units;
    a.nunits = t.nunits;
    a.counter = counter;
    a.stride = 0;
    a.boys = dev_boys();
    a.tabs = dev_class_tables();
    a.mt = nullptr;
    a.fp32_cutoff = Df ? fp32_cutoff : 0.0;
    a.fp32_cutoff_f = (float)a.fp32_cutoff;
    a.Df = Df;
    a.boysf = dev_boys_f();
    set_screen_args(a, tau, Dshf, prim_eps, cp);
    return launch_reg(t.reg_cb, t.reg_ck, a, t.blocks, 32 * t.warps_per_block, st);
  }
  cudaError_t ae = set_group_smem(t);
  if (ae != cudaSuccess) return ae;
  KArgs a;
  a.dp = dp;
  a.nprimtot = dp.nprim_total;
  a.nEtot = dp.nE_total;
  a.D = D;
  a.Dsh = Dsh;
  a.tau = tau;
  a.J = J;
  a.K = K;
  a.units = t.d_units;
  a.nunits = t.nunits;
  a.counter = counter;
  a.stride = t.stride;
  a.boys = dev_boys();
  a.tabs = dev_class_tables();
  a.mt = nullptr;
  a.fp32_cutoff = Df ? fp32_cutoff : 0.0;
  a.fp32_cutoff_f = (float)a.fp32_cutoff;
  a.Df = Df;
  a.boysf = dev_boys_f();
  set_screen_args(a, tau, Dshf, prim_eps, cp);
  return launch_group(t, a, 32 * t.warps_per_block, st, counter2);
}

// One tier of a batched build: same kernels, per-molecule D/J/K from mt.
cudaError_t launch_jk_tier_batch(const Tier &t, const DevPairs &dp, const MolEntry *mt, const double *Dsh,
                                 const float *Dshf, double tau, double prim_eps, int *counter, int *counter2,
                                 cudaStream_t st, double fp32_cutoff) {
  if (t.nunits == 0) return cudaSuccess;
  KArgs a;
  memset(&a, 0, sizeof(a));
  a.dp = dp;
  a.nprimtot = dp.nprim_total;
  a.nEtot = dp.nE_total;
  a.Dsh = Dsh;
  a.tau = tau;
  a.units = t.d_units;
  a.nunits = t.nunits;
  a.counter = counter;
  a.stride = t.stride;
  a.boys = dev_boys();
  a.tabs = dev_class_tables();
  a.boysf = dev_boys_f();
  a.mt = mt;
  a.fp32_cutoff = fp32_cutoff;
  a.fp32_cutoff_f = (float)a.fp32_cutoff;
  set_screen_args(a, tau, Dshf, prim_eps);
  const int threads = 32 * t.warps_per_block;
  if (t.reg_cb >= 0) {
    return launch_reg(t.reg_cb, t.reg_ck, a, t.blocks, threads, st);
  }
  cudaError_t ae = set_group_smem(t);
  if (ae != cudaSuccess) return ae;
  return launch_group(t, a, threads, st, counter2);
}

int read_bounds(long long out[2]) {
  return (int)cudaMemcpyFromSymbol(out, g_bounds, 2 * sizeof(long long));
}

int read_and_clear_status(cudaStream_t st, int *status) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return (int)e;
  int v = 0, zero = 0;
  e = cudaMemcpyFromSymbol(&v, g_status, sizeof(int));
  if (e != cudaSuccess) return (int)e;
  e = cudaMemcpyToSymbol(g_status, &zero, sizeof(int));
  if (e != cudaSuccess) return (int)e;
  *status = v;
  return 0;
}

}  // namespace fk
