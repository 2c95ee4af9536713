// FP64 one-electron integrals over the same normalised Cartesian basis:
// overlap S, kinetic T and nuclear attraction V (the core Hamiltonian
// h = T + V of Sec. 2.2, Eq. fock_build), by the McMurchie-Davidson Hermite
// expansion (Sec. 4.1, Eqs. EabP def1-3):
//   S_ab = sum_prims U_P E^{ab}_{000}
//   T_ab = -1/2 sum_x [4 b^2 S_x(a, b+2) - 2b(2 b_x + 1) S_x(a, b) + b_x(b_x - 1) S_x(a, b-2)] S_y S_z
//   V_ab = -sum_C Z_C sum_prims U_P 2 sqrt(zeta/pi) sum_tuv E^{ab}_tuv R_tuv(zeta, P - C)
// with U_P = c_a c_b (pi/zeta)^{3/2} exp(-a b |AB|^2 / zeta) and R seeded by
// (-2 zeta)^n F_n(zeta |P - C|^2).  One thread per (shell pair, Cartesian
// pair); all ordered shell pairs, so S, T, V come out full and symmetric.
#include <math.h>

#include <vector>

#include "device_common.cuh"

namespace fk {
fock_status validate_basis(const fock_basis_desc *d);
void normalised_coefs(const fock_basis_desc *d, int s, double *out);

namespace {

struct OneArgs {
  int nshell, nbf, natom;
  const double *xyz;    // shell centres
  const int *l, *np, *po, *bf;
  const double *ex, *cc;  // exponents, normalised coefficients
  const double *axyz, *Z;  // nuclei
  const double *boys;
  double *S, *T, *V;
};

// 1-D Hermite coefficients E^{ij}_t for i <= la, j <= lb (lb <= LMAX + 2)
__device__ void herm1d(int la, int lb, double p, double xpa, double xpb, double E[LMAX + 1][LMAX + 3][2 * LMAX + 4]) {
  const double h = 0.5 / p;
  for (int i = 0; i <= la; ++i)
    for (int j = 0; j <= lb; ++j)
      for (int t = 0; t <= i + j + 1; ++t) E[i][j][t] = 0.0;
  E[0][0][0] = 1.0;
  for (int i = 0; i < la; ++i)
    for (int t = 0; t <= i + 1; ++t) {
      double v = t <= i ? xpa * E[i][0][t] : 0.0;
      if (t > 0) v += h * E[i][0][t - 1];
      if (t + 1 <= i) v += (t + 1) * E[i][0][t + 1];
      E[i + 1][0][t] = v;
    }
  for (int i = 0; i <= la; ++i)
    for (int j = 0; j < lb; ++j)
      for (int t = 0; t <= i + j + 1; ++t) {
        double v = t <= i + j ? xpb * E[i][j][t] : 0.0;
        if (t > 0) v += h * E[i][j][t - 1];
        if (t + 1 <= i + j) v += (t + 1) * E[i][j][t + 1];
        E[i][j + 1][t] = v;
      }
}

__device__ double cart_norm_d(int x, int y, int z) {
  auto df = [](int n) {
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
  };
  return rsqrt(df(2 * x - 1) * df(2 * y - 1) * df(2 * z - 1));
}

__global__ void k_one_electron(OneArgs a) {
  const long long npairs = (long long)a.nshell * a.nshell;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // 100 Cartesian pairs per shell pair at most; one thread each
  const long long sp = tid / 100;
  const int kc = (int)(tid % 100);
  if (sp >= npairs) return;
  const int sa = (int)(sp / a.nshell), sb = (int)(sp % a.nshell);
  const int la = a.l[sa], lb = a.l[sb];
  const int nb = ncart(lb);
  if (kc >= ncart(la) * nb) return;
  int ax, ay, az, bx, by, bz;
  cart_comp(la, kc / nb, ax, ay, az);
  cart_comp(lb, kc % nb, bx, by, bz);
  const int av[3] = {ax, ay, az}, bv[3] = {bx, by, bz};
  const double *A = a.xyz + 3 * sa, *B = a.xyz + 3 * sb;
  double AB2 = 0.0;
  for (int x = 0; x < 3; ++x) AB2 += (A[x] - B[x]) * (A[x] - B[x]);
  double Ex[3][LMAX + 1][LMAX + 3][2 * LMAX + 4];
  double s = 0.0, t = 0.0, v = 0.0;
  for (int i = 0; i < a.np[sa]; ++i)
    for (int j = 0; j < a.np[sb]; ++j) {
      const double al = a.ex[a.po[sa] + i], be = a.ex[a.po[sb] + j], p = al + be;
      const double U = a.cc[a.po[sa] + i] * a.cc[a.po[sb] + j] * pow(3.141592653589793 / p, 1.5) * exp(-al * be / p * AB2);
      double P[3];
      for (int x = 0; x < 3; ++x) {
        P[x] = (al * A[x] + be * B[x]) / p;
        herm1d(av[x], bv[x] + 2, p, P[x] - A[x], P[x] - B[x], Ex[x]);
      }
      const double sx = Ex[0][ax][bx][0], sy = Ex[1][ay][by][0], sz = Ex[2][az][bz][0];
      s += U * sx * sy * sz;
      // kinetic: per direction -1/2 <a| d^2/dx^2 |b>
      double tk = 0.0;
      for (int x = 0; x < 3; ++x) {
        const int b = bv[x];
        double d2 = 4.0 * be * be * Ex[x][av[x]][b + 2][0] - 2.0 * be * (2 * b + 1) * Ex[x][av[x]][b][0];
        if (b >= 2) d2 += b * (b - 1) * Ex[x][av[x]][b - 2][0];
        const double o = (x == 0 ? sy * sz : (x == 1 ? sx * sz : sx * sy));
        tk += -0.5 * d2 * o;
      }
      t += U * tk;
      // nuclear attraction
      const int L = la + lb;
      const double pref = U * 2.0 * sqrt(p / 3.141592653589793);
      for (int c = 0; c < a.natom; ++c) {
        const double X = P[0] - a.axyz[3 * c], Y = P[1] - a.axyz[3 * c + 1], Zc = P[2] - a.axyz[3 * c + 2];
        const double T = p * (X * X + Y * Y + Zc * Zc);
        double F[2 * LMAX + 1];
        boys_eval_all(a.boys, L, T, F);
        // R^{(n)}_{tuv}: levels in place, R[n][e]
        double R[2 * LMAX + 1][nherm(2 * LMAX)];
        double c0 = 1.0;
        for (int n = 0; n <= L; ++n) {
          R[n][0] = c0 * F[n];
          c0 *= -2.0 * p;
        }
        for (int n = L - 1; n >= 0; --n)
          for (int e = 1; e < nherm(L - n); ++e) {
            int tt = 0, uu = 0, vv = 0, d = 0, k = 0;
            while (nherm(d) <= e) ++d;
            int r = e - (d > 0 ? nherm(d - 1) : 0);
            while (r > k) {
              r -= k + 1;
              ++k;
            }
            tt = d - k;
            uu = k - r;
            vv = r;
            double val;
            if (tt > 0) {
              val = X * R[n + 1][hidx(tt - 1, uu, vv)];
              if (tt > 1) val += (tt - 1) * R[n + 1][hidx(tt - 2, uu, vv)];
            } else if (uu > 0) {
              val = Y * R[n + 1][hidx(tt, uu - 1, vv)];
              if (uu > 1) val += (uu - 1) * R[n + 1][hidx(tt, uu - 2, vv)];
            } else {
              val = Zc * R[n + 1][hidx(tt, uu, vv - 1)];
              if (vv > 1) val += (vv - 1) * R[n + 1][hidx(tt, uu, vv - 2)];
            }
            R[n][e] = val;
          }
        double acc = 0.0;
        for (int tt = 0; tt <= ax + bx; ++tt)
          for (int uu = 0; uu <= ay + by; ++uu)
            for (int vv = 0; vv <= az + bz; ++vv)
              acc += Ex[0][ax][bx][tt] * Ex[1][ay][by][uu] * Ex[2][az][bz][vv] * R[0][hidx(tt, uu, vv)];
        v -= a.Z[c] * pref * acc;
      }
    }
  const double f = cart_norm_d(ax, ay, az) * cart_norm_d(bx, by, bz);
  const size_t o = (size_t)(a.bf[sa] + kc / nb) * a.nbf + a.bf[sb] + kc % nb;
  a.S[o] = f * s;
  a.T[o] = f * t;
  a.V[o] = f * v;
}

}  // namespace
}  // namespace fk

using namespace fk;

extern "C" fock_status fock_one_electron(const fock_basis_desc *desc, int32_t natom, const double *Z,
                                         const double *xyz, double *S, double *T, double *V, cudaStream_t stream) {
  fock_status vs = validate_basis(desc);
  if (vs != FOCK_OK) return vs;
  if (natom < 0 || (natom > 0 && (!Z || !xyz)) || !S || !T || !V) return FOCK_ERR_INVALID_ARG;
  cudaError_t e = upload_tables(stream);
  if (e != cudaSuccess) return FOCK_ERR_CUDA;
  const int ns = desc->nshell;
  int np_tot = 0;
  std::vector<int> bf(ns), l(desc->l, desc->l + ns), np(desc->nprim, desc->nprim + ns), po(ns);
  int nbf = 0;
  for (int s = 0; s < ns; ++s) {
    bf[s] = nbf;
    nbf += ncart(l[s]);
    po[s] = np_tot;
    np_tot += np[s];
  }
  std::vector<double> ex(np_tot), cc(np_tot), c(desc->center, desc->center + 3 * ns);
  for (int s = 0; s < ns; ++s) {
    normalised_coefs(desc, s, cc.data() + po[s]);
    for (int i = 0; i < np[s]; ++i) ex[po[s] + i] = desc->exps[desc->prim_off[s] + i];
  }
  // one device block for every input array
  const size_t nb_i = sizeof(int) * 4 * ns, nb_d = sizeof(double) * (3 * ns + 2 * np_tot + 4 * natom + 4);
  char *d = nullptr;
  e = cudaMallocAsync((void **)&d, nb_i + nb_d, stream);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FOCK_ERR_OOM : FOCK_ERR_CUDA;
  std::vector<char> host(nb_i + nb_d);
  int *hi = (int *)host.data();
  memcpy(hi, l.data(), sizeof(int) * ns);
  memcpy(hi + ns, np.data(), sizeof(int) * ns);
  memcpy(hi + 2 * ns, po.data(), sizeof(int) * ns);
  memcpy(hi + 3 * ns, bf.data(), sizeof(int) * ns);
  double *hd = (double *)(host.data() + nb_i);
  memcpy(hd, c.data(), sizeof(double) * 3 * ns);
  memcpy(hd + 3 * ns, ex.data(), sizeof(double) * np_tot);
  memcpy(hd + 3 * ns + np_tot, cc.data(), sizeof(double) * np_tot);
  if (natom > 0) {
    memcpy(hd + 3 * ns + 2 * np_tot, xyz, sizeof(double) * 3 * natom);
    memcpy(hd + 3 * ns + 2 * np_tot + 3 * natom, Z, sizeof(double) * natom);
  }
  e = cudaMemcpyAsync(d, host.data(), nb_i + nb_d, cudaMemcpyHostToDevice, stream);
  OneArgs a;
  const int *di = (const int *)d;
  const double *dd = (const double *)(d + nb_i);
  a.nshell = ns;
  a.nbf = nbf;
  a.natom = natom;
  a.l = di;
  a.np = di + ns;
  a.po = di + 2 * ns;
  a.bf = di + 3 * ns;
  a.xyz = dd;
  a.ex = dd + 3 * ns;
  a.cc = dd + 3 * ns + np_tot;
  a.axyz = dd + 3 * ns + 2 * np_tot;
  a.Z = dd + 3 * ns + 2 * np_tot + 3 * natom;
  a.boys = dev_boys();
  a.S = S;
  a.T = T;
  a.V = V;
  if (e == cudaSuccess) {
    const long long nthr = (long long)ns * ns * 100;
    k_one_electron<<<(unsigned)((nthr + 127) / 128), 128, 0, stream>>>(a);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(d, stream);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  return e == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA;
}
