// Device helpers shared by the J/K kernels.
//
// GB300 issues FP64 instructions at 1/64 of the FP32 rate, while integer and
// FP32 work is plentiful.  These helpers therefore move everything that does
// not need 53-bit precision (grid indices, branch decisions, initial
// approximations) to FP32/integer units and keep the FP64 instruction count
// per primitive quartet small.
#pragma once

#include "fock_impl.h"

namespace fk {

// Exact float -> double by bit manipulation on the integer units (valid for
// positive normal floats, which is all it is used for).
__device__ __forceinline__ double f2d_pos(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long e = ((u >> 23) & 0xffu) + (1023u - 127u);
  const unsigned long long m = u & 0x7fffffu;
  return __longlong_as_double((long long)((e << 52) | (m << 29)));
}

// Exact float -> double on the integer units for any finite float
// (zero and subnormal inputs map to 0, |x| < 1.2e-38).
__device__ __forceinline__ double f2d_any(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0) return 0.0;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned long long e = ex + (1023u - 127u);
  const unsigned long long m = u & 0x7fffffu;
  return __longlong_as_double((long long)(sign | (e << 52) | (m << 29)));
}

// 1/sqrt(s) for s > 0 in double precision: FP32 seed y0 = rsqrtf(s_f), then
// one third-order Householder step of the Newton iteration for 1/sqrt
// (error e = 1 - s y0^2, y = y0 (1 + e/2 + 3e^2/8)); the seed's relative
// error ~3e-7 is cubed to ~3e-20, so the result is limited by FP64 rounding.
// sf is s rounded to FP32 (computed by the caller on the FP32 units).
__device__ __forceinline__ double rsqrt_nh(double s, float sf) {
  const double y0 = f2d_pos(rsqrtf(sf));
  const double t = s * y0;
  const double e = fma(-t, y0, 1.0);
  const double c = e * fma(e, 0.375, 0.5);
  return fma(y0, c, y0);
}

// Quantities of one primitive quartet [ab|cd] used by every class.
struct PrimQuartet {
  double X, Y, Z;   // P - Q
  double T;         // alpha |P - Q|^2
  double m2a;       // -2 alpha
  double pref;      // 1/sqrt(zeta + eta); the pair factors U_P sqrt(zeta) (2/sqrt(pi))^(1/2)
                    // are folded into the Hermite coefficients, so pref times them is
                    // U_P U_Q 2 sqrt(alpha/pi)
  int gi;           // Boys grid index (T < BOYS_TMAX) or -1 (asymptotic)
  double Ti;        // grid abscissa i*h (exact)
  float Tf;         // T on the FP32 units (seed of the asymptotic rsqrt)
};

// P4 = (Px, Py, Pz, zeta), Pf = the same in FP32.
__device__ __forceinline__ PrimQuartet prim_quartet(const PZ &P4, const float4 &Pf, const PZ &Q4,
                                                    const float4 &Qf) {
  PrimQuartet r;
  const double s = P4.w + Q4.w;
  const float sf = Pf.w + Qf.w;
  const double rs = rsqrt_nh(s, sf);
  r.pref = rs;
  const double alpha = (P4.w * Q4.w) * (rs * rs);
  r.m2a = -2.0 * alpha;
  r.X = P4.x - Q4.x;
  r.Y = P4.y - Q4.y;
  r.Z = P4.z - Q4.z;
  r.T = alpha * fma(r.X, r.X, fma(r.Y, r.Y, r.Z * r.Z));
  // grid decision on the FP32 units (an index off by one at a half-point
  // still leaves |T - T_i| < h, well inside the Taylor error bound)
  const float xf = Pf.x - Qf.x, yf = Pf.y - Qf.y, zf = Pf.z - Qf.z;
  const float Tf = __fdividef(Pf.w * Qf.w, sf) * (xf * xf + yf * yf + zf * zf);
  r.Tf = Tf;
  if (Tf < (float)BOYS_TMAX) {
    r.gi = __float2int_rn(Tf * (float)BOYS_INVH);
    r.Ti = (r.gi == 0) ? 0.0 : f2d_pos((float)r.gi * (float)BOYS_H);
  } else {
    r.gi = -1;
    r.Ti = 0.0;
  }
  return r;
}

// F_m(T) for one m from the table (Taylor about T_i, Horner in x = T_i - T).
// The eight coefficients of an entry are 64 contiguous bytes on a 64-byte
// boundary (the table is one device allocation), read as four 16-byte loads.
__device__ __forceinline__ double boys_taylor(const double *__restrict__ tab, int gi, int m, double x) {
  const double2 *c = reinterpret_cast<const double2 *>(tab + ((size_t)gi * (LTOT + 1) + m) * BOYS_TAYLOR);
  const double2 c67 = __ldg(c + 3), c45 = __ldg(c + 2), c23 = __ldg(c + 1), c01 = __ldg(c);
  double f = fma(c67.y, x, c67.x);
  f = fma(f, x, c45.y);
  f = fma(f, x, c45.x);
  f = fma(f, x, c23.y);
  f = fma(f, x, c23.x);
  f = fma(f, x, c01.y);
  return fma(f, x, c01.x);
}

// x rounded toward zero to FP32 on the integer units (|x| < 2^-126 gives 0);
// used for the Taylor variable, |x| <= h/2.
__device__ __forceinline__ float d2f_small(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return 0.0f;
  const unsigned sign = (unsigned)(u >> 63) << 31;
  return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((u >> 29) & 0x7fffffu));
}

// The same Taylor polynomial with its four highest terms on the FP32 units:
// with |x| <= h/2 = 1/32 and F_{m+k} <= F_m, the terms k >= 4 add at most
// (1/32)^4/4! F_m = 4e-8 F_m, so their FP32 rounding (and the FP32 copies of
// c4..c7 and of x) perturbs F_m by about 1e-14 relative, while four FP64
// fused multiply-adds are saved per order.  tabf is the FP32 copy of the
// table (same layout); c4..c7 are its entry's second 16 bytes.
__device__ __forceinline__ double boys_taylor_split(const double *__restrict__ tab, const float *__restrict__ tabf,
                                                    int gi, int m, double x, float xf) {
  const size_t ent = ((size_t)gi * (LTOT + 1) + m) * BOYS_TAYLOR;
  const double2 *c = reinterpret_cast<const double2 *>(tab + ent);
  const double2 c23 = __ldg(c + 1), c01 = __ldg(c);
  const float4 h = __ldg(reinterpret_cast<const float4 *>(tabf + ent) + 1);
  float t = fmaf(h.w, xf, h.z);
  t = fmaf(t, xf, h.y);
  t = fmaf(t, xf, h.x);
  double f = fma(f2d_any(t), x, c23.y);
  f = fma(f, x, c23.x);
  f = fma(f, x, c01.y);
  return fma(f, x, c01.x);
}

// Seeds pref (-2 alpha)^m F_m(T), m = 0..L, into out[] (compile-time L);
// tabf (the FP32 table) selects the split evaluation.
template <int L>
__device__ __forceinline__ void boys_seeds(const double *__restrict__ tab, const PrimQuartet &q, double (&out)[L + 1],
                                           const float *__restrict__ tabf = nullptr) {
  if (q.gi >= 0) {
    const double x = q.Ti - q.T;
    if (tabf) {
      const float xf = d2f_small(x);
#pragma unroll
      for (int m = 0; m <= L; ++m) out[m] = boys_taylor_split(tab, tabf, q.gi, m, x, xf);
    } else {
#pragma unroll
      for (int m = 0; m <= L; ++m) out[m] = boys_taylor(tab, q.gi, m, x);
    }
  } else {
    // asymptotic: F_0 = sqrt(pi/T)/2, F_m = F_{m-1} (m - 1/2) / T
    const double rt = rsqrt_nh(q.T, q.Tf);
    out[0] = 0.88622692545275801365 * rt;  // sqrt(pi)/2
    const double it = rt * rt;
#pragma unroll
    for (int m = 1; m <= L; ++m) out[m] = out[m - 1] * ((m - 0.5) * it);
  }
  double c = q.pref;
#pragma unroll
  for (int m = 0; m <= L; ++m) {
    out[m] *= c;
    c *= q.m2a;
  }
}

// F_m(T), m = 0..L (no seed scaling), full FP64 (one-electron integrals).
__device__ __forceinline__ void boys_eval_all(const double *__restrict__ tab, int L, double T, double *F) {
  if (T < BOYS_TMAX) {
    const int gi = (int)(T * BOYS_INVH + 0.5);
    const double x = gi * BOYS_H - T;
    for (int m = 0; m <= L; ++m) F[m] = boys_taylor(tab, gi, m, x);
  } else {
    F[0] = 0.88622692545275801365 * rsqrt(T);
    const double it = 1.0 / T;
    for (int m = 1; m <= L; ++m) F[m] = F[m - 1] * (m - 0.5) * it;
  }
}

// Runtime-L variant for the group-cooperative kernel: lanes gl, gl+G, ...
// write seeds m into F[]; the lane that writes m = L also writes R0[0].
template <int G>
__device__ __forceinline__ void boys_seeds_rt(const double *__restrict__ tab, const PrimQuartet &q, int L, double *F,
                                              double *R0, int gl, const float *__restrict__ tabf = nullptr) {
  if constexpr (G == 1) {
    double c = q.pref, prev = 0.0;
    const double x = q.Ti - q.T;
    const float xf = d2f_small(x);
    double rt = 0.0, it = 0.0;
    if (q.gi < 0) {
      rt = rsqrt_nh(q.T, q.Tf);
      it = rt * rt;
    }
    for (int m = 0; m <= L; ++m) {
      double f;
      if (q.gi >= 0)
        f = tabf ? boys_taylor_split(tab, tabf, q.gi, m, x, xf) : boys_taylor(tab, q.gi, m, x);
      else
        f = (m == 0) ? 0.88622692545275801365 * rt : prev * ((m - 0.5) * it);
      prev = f;
      F[m] = f * c;
      c *= q.m2a;
    }
    R0[0] = F[L];
  } else {
  for (int m = gl; m <= L; m += G) {
    double f;
    if (q.gi >= 0) {
      const double x = q.Ti - q.T;
      f = tabf ? boys_taylor_split(tab, tabf, q.gi, m, x, d2f_small(x)) : boys_taylor(tab, q.gi, m, x);
    } else {
      const double rt = rsqrt_nh(q.T, q.Tf), it = rt * rt;
      f = 0.88622692545275801365 * rt;
      for (int k = 1; k <= m; ++k) f *= (k - 0.5) * it;
    }
    double c = q.pref;
    for (int k = 0; k < m; ++k) c *= q.m2a;
    F[m] = f * c;
    if (m == L) R0[0] = F[m];
  }
  }
}


// FP32 seeds pref (-2 alpha)^m F_m(T), m = 0..L: six Taylor terms from the
// FP32 copy of the table (truncation < 2e-12 relative) or the asymptotic form.
template <int L>
__device__ __forceinline__ void boys_seeds_f32(const float *__restrict__ tab, float T, float pref, float m2a,
                                               float (&out)[L + 1]) {
  if (T < (float)BOYS_TMAX) {
    const int gi = __float2int_rn(T * (float)BOYS_INVH);
    const float x = (float)gi * (float)BOYS_H - T;
#pragma unroll
    for (int m = 0; m <= L; ++m) {
      // six of the entry's eight coefficients (32 bytes on a 32-byte boundary)
      const float4 *c = reinterpret_cast<const float4 *>(tab + ((size_t)gi * (LTOT + 1) + m) * BOYS_TAYLOR);
      const float4 c03 = __ldg(c);
      const float2 c45 = __ldg(reinterpret_cast<const float2 *>(c + 1));
      float f = fmaf(c45.y, x, c45.x);
      f = fmaf(f, x, c03.w);
      f = fmaf(f, x, c03.z);
      f = fmaf(f, x, c03.y);
      out[m] = fmaf(f, x, c03.x);
    }
  } else {
    const float rt = rsqrtf(T);
    out[0] = 0.886226925452758f * rt;
    const float it = rt * rt;
#pragma unroll
    for (int m = 1; m <= L; ++m) out[m] = out[m - 1] * ((m - 0.5f) * it);
  }
  float c = pref;
#pragma unroll
  for (int m = 0; m <= L; ++m) {
    out[m] *= c;
    c *= m2a;
  }
}

}  // namespace fk
