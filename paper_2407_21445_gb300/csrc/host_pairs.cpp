// Host-side precomputation of the J/K builder: Boys table, class tables,
// normalisation, primitive pairs with Hermite expansion coefficients, pair
// pruning, binning and the quartet work units.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "fock_impl.h"

namespace fk {

// --------------------------------------------------------------------------
// Boys function table (Eq. boys-fn-def): each order by its own power series
//   F_k(T) = exp(-T) sum_j (2T)^j / ((2k+1)(2k+3)...(2k+2j+1)),
// stored as Taylor coefficients F_{m+k}(T_i)/k! about T_i = i h.
// --------------------------------------------------------------------------
static double boys_series(int k, double T) {
  double term = 1.0 / (2.0 * k + 1.0), sum = term;
  for (int j = 1; j < 4000; ++j) {
    term *= 2.0 * T / (2.0 * k + 2.0 * j + 1.0);
    sum += term;
    if (term < 1e-19 * sum) break;
  }
  return exp(-T) * sum;
}

const std::vector<double> &boys_table() {
  static std::vector<double> tab;
  static std::once_flag once;
  std::call_once(once, [] {
    tab.assign((size_t)BOYS_NGRID * (LTOT + 1) * BOYS_TAYLOR, 0.0);
    double fact[BOYS_TAYLOR];
    fact[0] = 1.0;
    for (int k = 1; k < BOYS_TAYLOR; ++k) fact[k] = fact[k - 1] * k;
    std::vector<double> F(BOYS_NORD);
    for (int i = 0; i < BOYS_NGRID; ++i) {
      const double T = i * BOYS_H;
      for (int k = 0; k < BOYS_NORD; ++k) F[k] = boys_series(k, T);
      for (int m = 0; m <= LTOT; ++m)
        for (int k = 0; k < BOYS_TAYLOR; ++k)
          tab[((size_t)i * (LTOT + 1) + m) * BOYS_TAYLOR + k] = F[m + k] / fact[k];
    }
  });
  return tab;
}

// Same rule as the device evaluator, on the host.
void boys_eval_host(int mmax, double T, double *F) {
  const std::vector<double> &tab = boys_table();
  for (int m = 0; m <= mmax; ++m) {
    if (T < BOYS_TMAX) {
      const int i = (int)nearbyint(T * BOYS_INVH);
      const double x = i * BOYS_H - T;
      const double *c = tab.data() + ((size_t)i * (LTOT + 1) + m) * BOYS_TAYLOR;
      double f = c[7];
      for (int k = 6; k >= 0; --k) f = fma(f, x, c[k]);
      F[m] = f;
    } else {
      double f = 0.5 * sqrt(M_PI / T);
      const double h = 0.5 / T;
      for (int k = 1; k <= m; ++k) f *= (2 * k - 1) * h;
      F[m] = f;
    }
  }
}

// --------------------------------------------------------------------------
// class tables
// --------------------------------------------------------------------------
const ClassTables &class_tables() {
  static ClassTables ct;
  static std::once_flag once;
  std::call_once(once, [] {
    memset(&ct, 0, sizeof(ct));
    for (int l = 0; l <= LMAX; ++l)
      for (int i = 0; i < ncart(l); ++i) {
        int x, y, z;
        cart_comp(l, i, x, y, z);
        ct.comp[l][i][0] = (uint8_t)x;
        ct.comp[l][i][1] = (uint8_t)y;
        ct.comp[l][i][2] = (uint8_t)z;
      }
    for (int d = 0; d <= LTOT; ++d)
      for (int t = d; t >= 0; --t)
        for (int u = d - t; u >= 0; --u) {
          const int v = d - t - u, e = hidx(t, u, v);
          ct.hvec[e][0] = (uint8_t)t;
          ct.hvec[e][1] = (uint8_t)u;
          ct.hvec[e][2] = (uint8_t)v;
        }
    for (int la = 0; la <= LMAX; ++la)
      for (int lb = 0; lb <= la; ++lb) {
        const int c = pair_class(la, lb);
        int off = 0, k = 0;
        for (int ia = 0; ia < ncart(la); ++ia)
          for (int ib = 0; ib < ncart(lb); ++ib, ++k) {
            ct.eoff[c][k] = (int16_t)off;
            off += (ct.comp[la][ia][0] + ct.comp[lb][ib][0] + 1) * (ct.comp[la][ia][1] + ct.comp[lb][ib][1] + 1) *
                   (ct.comp[la][ia][2] + ct.comp[lb][ib][2] + 1);
          }
        ct.eoff[c][k] = (int16_t)off;
        ct.nE[c] = (int16_t)off;
      }
  });
  return ct;
}

int hermite_count(int la, int lb) {
  int n = 0;
  for (int ia = 0; ia < ncart(la); ++ia)
    for (int ib = 0; ib < ncart(lb); ++ib) {
      int ax, ay, az, bx, by, bz;
      cart_comp(la, ia, ax, ay, az);
      cart_comp(lb, ib, bx, by, bz);
      n += (ax + bx + 1) * (ay + by + 1) * (az + bz + 1);
    }
  return n;
}

// 1-D Hermite expansion coefficients (Sec. 4.1, Eqs. EabP def1-3):
// E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1},
// E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1},
// E^{00}_0 = 1 (the Gaussian-product prefactor K_AB is kept in U_P).
// Layout E[(i*4 + j)*7 + t].
void hermite_1d(int la, int lb, double p, double xpa, double xpb, double *E) {
  memset(E, 0, sizeof(double) * 4 * 4 * 7);
  const double h = 0.5 / p;
  E[0] = 1.0;
  for (int i = 0; i < la; ++i)
    for (int t = 0; t <= i + 1; ++t) {
      double v = xpa * (t <= i ? E[(i * 4) * 7 + t] : 0.0);
      if (t > 0) v += h * E[(i * 4) * 7 + t - 1];
      if (t + 1 <= i) v += (t + 1) * E[(i * 4) * 7 + t + 1];
      E[((i + 1) * 4) * 7 + t] = v;
    }
  for (int i = 0; i <= la; ++i)
    for (int j = 0; j < lb; ++j)
      for (int t = 0; t <= i + j + 1; ++t) {
        const double *src = E + (i * 4 + j) * 7;
        double v = xpb * (t <= i + j ? src[t] : 0.0);
        if (t > 0) v += h * src[t - 1];
        if (t + 1 <= i + j) v += (t + 1) * src[t + 1];
        E[(i * 4 + j + 1) * 7 + t] = v;
      }
}

static double dfact(int n) {
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

static double cart_norm(int x, int y, int z) { return 1.0 / sqrt(dfact(2 * x - 1) * dfact(2 * y - 1) * dfact(2 * z - 1)); }

void hermite_pair(int la, int lb, double alpha, const double *A, double beta, const double *B, bool cnorm,
                  double *out) {
  const double p = alpha + beta;
  double E[3][4 * 4 * 7];
  for (int x = 0; x < 3; ++x) {
    const double P = (alpha * A[x] + beta * B[x]) / p;
    hermite_1d(la, lb, p, P - A[x], P - B[x], E[x]);
  }
  int o = 0;
  for (int ia = 0; ia < ncart(la); ++ia)
    for (int ib = 0; ib < ncart(lb); ++ib) {
      int ax, ay, az, bx, by, bz;
      cart_comp(la, ia, ax, ay, az);
      cart_comp(lb, ib, bx, by, bz);
      const double f = cnorm ? cart_norm(ax, ay, az) * cart_norm(bx, by, bz) : 1.0;
      const double *ex = E[0] + (ax * 4 + bx) * 7, *ey = E[1] + (ay * 4 + by) * 7, *ez = E[2] + (az * 4 + bz) * 7;
      for (int t = 0; t <= ax + bx; ++t)
        for (int u = 0; u <= ay + by; ++u)
          for (int v = 0; v <= az + bz; ++v) out[o++] = f * ex[t] * ey[u] * ez[v];
    }
}

}  // namespace fk
