// C-ABI entry points of the J/K builder (declared in include/fock.h) and the
// shell-pair handle construction.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include "fock_impl.h"
#include "kernels_reg.cuh"
#include "reg_dispatch.h"

using namespace fk;

namespace {

constexpr double kPi = 3.141592653589793238462643383;


// Device copy of a Staging set plus units: one allocation, 256-byte aligned
// sub-buffers.  Returns the base pointer; fills dp and unit pointers.
struct Packer {
  size_t off = 0;
  std::vector<std::pair<size_t, std::pair<const void *, size_t>>> parts;
  size_t add(const void *src, size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    size_t at = off;
    parts.push_back({at, {src, bytes}});
    off += bytes;
    return at;
  }
};

thread_local char g_last_error[256] = "";

fock_status to_status(cudaError_t e, const char *where = "cuda") {
  if (e == cudaSuccess) return FOCK_OK;
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return FOCK_ERR_OOM;
  return FOCK_ERR_CUDA;
}

bool sync_check() {
  static int v = -1;
  if (v < 0) {
    const char *s = getenv("FOCK_SYNC_CHECK");
    v = (s && s[0] == '1') ? 1 : 0;
  }
  return v == 1;
}

// Scratch (doubles) one group needs for a quartet of bra class cb, ket class ck.
int scratch_doubles(int la, int lb, int lc, int ld) {
  const int nab = ncart(la) * ncart(lb), ncd = ncart(lc) * ncart(ld);
  const int Lab = la + lb, L = la + lb + lc + ld;
  return nab * ncd + nherm(Lab) * ncd + 2 * nherm(L) + L + 2;
}

void class_l(int c, int &la, int &lb) {
  la = 0;
  while ((la + 1) * (la + 2) / 2 <= c) ++la;
  lb = c - la * (la + 1) / 2;
}

// FP64 operation model (an FMA counts 2) of one primitive quartet (Boys
// Taylor, seeds, R recursion, ket transform) and per bra primitive (bra
// transform).  Per primitive quartet: zeta + eta 1, 1/sqrt by one Newton-
// Householder step 8, alpha 3, -2 alpha 1, P - Q 3, T 6, T_i - T 1 = 23;
// per Boys order 4 FP64 Horner FMAs 8 (the four highest Taylor terms run on
// the FP32 units and are not counted), seed scaling 1, power of -2 alpha 1
// = 10.
double flops_prim(int Lab, int L, int ck) {
  const ClassTables &ct = class_tables();
  double f = 23.0;                  // alpha, T, 1/sqrt(zeta + eta)
  f += (L + 1) * 10.0;              // Taylor Horner + seed scaling
  for (int n = L - 1; n >= 0; --n)  // Hermite recursion
    for (int e = 1; e < nherm(L - n); ++e) {
      const int t = ct.hvec[e][0], u = ct.hvec[e][1], w = ct.hvec[e][2];
      const int c = t > 0 ? t : (u > 0 ? u : w);
      f += c > 1 ? 3.0 : 1.0;
    }
  f += 2.0 * nherm(Lab) * ct.nE[ck];
  return f;
}

double flops_bra(int cb, int ncd) { return 2.0 * class_tables().nE[cb] * ncd; }

// flops_prim / flops_bra per (bra class, ket class), cached
struct FlopTable {
  double prim[NCLASS][NCLASS], bra[NCLASS][NCLASS];
  FlopTable() {
    for (int cb = 0; cb < NCLASS; ++cb)
      for (int ck = 0; ck < NCLASS; ++ck) {
        int la, lb, lc, ld;
        class_l(cb, la, lb);
        class_l(ck, lc, ld);
        prim[cb][ck] = flops_prim(la + lb, la + lb + lc + ld, ck);
        bra[cb][ck] = flops_bra(cb, ncart(lc) * ncart(ld));
      }
  }
};
const FlopTable &flop_table() {
  static FlopTable t;
  return t;
}

// Contraction bins: pairs with the same number of kept primitive pairs share
// a bin up to 16, then bins 4 wide, so that the 32 kets a warp takes have
// nearly equal primitive loops (lanes of a warp wait for the longest).
constexpr bool kFineBins = true;
int bucket_of(int nprim) {
  if (kFineBins) return nprim <= 16 ? nprim : 16 + (nprim - 13) / 4;
  int b = 0;
  while ((1 << b) < nprim) ++b;
  return b;  // 1 -> 0, 2 -> 1, 3..4 -> 2, 5..8 -> 3, ...
}

fock_status validate(const fock_basis_desc *d) {
  if (!d || d->nshell < 1 || !d->center || !d->l || !d->nprim || !d->prim_off || !d->exps || !d->coefs)
    return FOCK_ERR_INVALID_ARG;
  for (int s = 0; s < d->nshell; ++s) {
    if (d->l[s] < 0 || d->l[s] > LMAX) return FOCK_ERR_UNSUPPORTED_L;
    if (d->nprim[s] < 1 || d->nprim[s] > MAXPRIM) return FOCK_ERR_UNSUPPORTED_L;
    if (d->prim_off[s] < 0) return FOCK_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
      if (!isfinite(d->center[3 * s + k])) return FOCK_ERR_INVALID_ARG;
    for (int i = 0; i < d->nprim[s]; ++i) {
      const double a = d->exps[d->prim_off[s] + i], c = d->coefs[d->prim_off[s] + i];
      if (!(a > 0.0) || !isfinite(a) || !isfinite(c)) return FOCK_ERR_INVALID_ARG;
    }
  }
  return FOCK_OK;
}

// Normalised contraction coefficients: raw coefficient x primitive factor
// (2a/pi)^{3/4} (4a)^{l/2} x contracted factor making every Cartesian
// function of unit norm (the component factor 1/sqrt(prod (2k-1)!!) is folded
// into the Hermite coefficients).
void norm_coefs(const fock_basis_desc *d, int s, double *out) {
  const int l = d->l[s], K = d->nprim[s], o = d->prim_off[s];
  double S = 0.0;
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) {
      const double ai = d->exps[o + i], aj = d->exps[o + j];
      S += d->coefs[o + i] * d->coefs[o + j] * pow(2.0 * sqrt(ai * aj) / (ai + aj), l + 1.5);
    }
  const double nc = 1.0 / sqrt(S);
  for (int i = 0; i < K; ++i) {
    const double a = d->exps[o + i];
    out[i] = nc * d->coefs[o + i] * pow(2.0 * a / kPi, 0.75) * pow(4.0 * a, 0.5 * l);
  }
}

fock_status upload(const Staging &st, const std::vector<Unit> &units, void **base, DevPairs &dp, Unit **d_units,
                   size_t *bytes, cudaStream_t stream) {
  Packer pk;
  const size_t o_sxyz = pk.add(st.sxyz.data(), st.sxyz.size() * sizeof(double));
  const size_t o_sbf = pk.add(st.sbf.data(), st.sbf.size() * sizeof(int));
  const size_t o_sl = pk.add(st.sl.data(), st.sl.size() * sizeof(int));
  const size_t o_ab = pk.add(st.ab.data(), st.ab.size() * sizeof(int2));
  const size_t o_G = pk.add(st.G.data(), st.G.size() * sizeof(double));
  const size_t o_prim = pk.add(st.prim.data(), st.prim.size() * sizeof(int2));
  const size_t o_cls = pk.add(st.cls.data(), st.cls.size() * sizeof(int));
  const size_t o_pz = pk.add(st.pz.data(), st.pz.size() * sizeof(PZ));
  const size_t o_pf = pk.add(st.pf.data(), st.pf.size() * sizeof(float4));
  const size_t o_U = pk.add(st.U.data(), st.U.size() * sizeof(double));
  const size_t o_eoff = pk.add(st.eoff.data(), st.eoff.size() * sizeof(int));
  const size_t o_E = pk.add(st.E.data(), st.E.size() * sizeof(double));
  const size_t o_Gp = pk.add(st.Gp.data(), st.Gp.size() * sizeof(double));
  const size_t o_Gpf = pk.add(st.Gpf.data(), st.Gpf.size() * sizeof(float));
  const size_t o_Gf = pk.add(st.Gf.data(), st.Gf.size() * sizeof(float));
  const size_t o_shl = pk.add(st.shl.data(), st.shl.size() * sizeof(float));
  const size_t o_paf = pk.add(st.paf.data(), st.paf.size() * sizeof(float4));
  const size_t o_Uf = pk.add(st.Uf.data(), st.Uf.size() * sizeof(float));
  const size_t o_Ef = pk.add(st.Ef.data(), st.Ef.size() * sizeof(float));
  const size_t o_smol = pk.add(st.smol.data(), st.smol.size() * sizeof(int));
  const size_t o_satom = pk.add(st.satom.data(), st.satom.size() * sizeof(int));
  const size_t o_sRG = pk.add(st.sRG.data(), st.sRG.size() * sizeof(float2));
  const size_t o_Gn = pk.add(st.Gn.data(), st.Gn.size() * sizeof(float));
  const size_t o_units = pk.add(units.data(), units.size() * sizeof(Unit));
  const size_t total = (pk.off + 255) & ~(size_t)255;
  char *d = nullptr;
  cudaError_t e = cudaMalloc(&d, total > 0 ? total : 256);
  if (e != cudaSuccess) return to_status(e);
  for (auto &p : pk.parts) {
    if (p.second.second == 0) continue;
    e = cudaMemcpyAsync(d + p.first, p.second.first, p.second.second, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) {
      cudaFree(d);
      return to_status(e);
    }
  }
  dp.sxyz = (const double *)(d + o_sxyz);
  dp.sbf = (const int *)(d + o_sbf);
  dp.sl = (const int *)(d + o_sl);
  dp.ab = (const int2 *)(d + o_ab);
  dp.G = (const double *)(d + o_G);
  dp.prim = (const int2 *)(d + o_prim);
  dp.cls = (const int *)(d + o_cls);
  dp.pz = (const PZ *)(d + o_pz);
  dp.pf = (const float4 *)(d + o_pf);
  dp.U = (const double *)(d + o_U);
  dp.eoff = (const int *)(d + o_eoff);
  dp.E = (const double *)(d + o_E);
  dp.Gp = st.Gp.empty() ? nullptr : (const double *)(d + o_Gp);
  dp.Gpf = st.Gpf.empty() ? nullptr : (const float *)(d + o_Gpf);
  dp.paf = (const float4 *)(d + o_paf);
  dp.Gf = (const float *)(d + o_Gf);
  dp.smol = st.smol.empty() ? nullptr : (const int *)(d + o_smol);
  dp.satom = st.satom.empty() ? nullptr : (const int *)(d + o_satom);
  dp.sRG = st.sRG.empty() ? nullptr : (const float2 *)(d + o_sRG);
  dp.Gn = st.Gn.empty() ? nullptr : (const float *)(d + o_Gn);
  dp.shl = (const float *)(d + o_shl);
  dp.Uf = (const float *)(d + o_Uf);
  dp.Ef = (const float *)(d + o_Ef);
  dp.npair = (int)st.ab.size();
  dp.nprim_total = (int)st.pz.size();
  dp.nE_total = (long long)st.E.size();
  if (d_units) *d_units = (Unit *)(d + o_units);
  *base = d;
  if (bytes) *bytes = total;
  return FOCK_OK;
}

}  // namespace

namespace fk {
fock_status cuda_status(cudaError_t e, const char *where) { return to_status(e, where); }
bool sync_each_launch() { return sync_check(); }
fock_status validate_basis(const fock_basis_desc *d) { return validate(d); }
void normalised_coefs(const fock_basis_desc *d, int s, double *out) { norm_coefs(d, s, out); }
fock_status upload_staging(const Staging &st, const std::vector<Unit> &units, void **base, DevPairs &dp,
                           Unit **d_units, size_t *bytes, cudaStream_t stream) {
  return upload(st, units, base, dp, d_units, bytes, stream);
}
}  // namespace fk

extern "C" {

const char *fock_last_error(void) { return g_last_error; }

fock_status fock_debug_bounds(int64_t out[2]) {
  if (!out) return FOCK_ERR_INVALID_ARG;
  long long v[2] = {0, 0};
  if (read_bounds(v)) return FOCK_ERR_CUDA;
  out[0] = v[0];
  out[1] = v[1];
  return FOCK_OK;
}

const char *fock_status_string(fock_status st) {
  switch (st) {
    case FOCK_OK: return "FOCK_OK";
    case FOCK_ERR_INVALID_ARG: return "FOCK_ERR_INVALID_ARG";
    case FOCK_ERR_UNSUPPORTED_L: return "FOCK_ERR_UNSUPPORTED_L";
    case FOCK_ERR_NONFINITE: return "FOCK_ERR_NONFINITE";
    case FOCK_ERR_OOM: return "FOCK_ERR_OOM";
    case FOCK_ERR_CUDA: return "FOCK_ERR_CUDA";
    case FOCK_ERR_TIMEOUT: return "FOCK_ERR_TIMEOUT";
    case FOCK_ERR_NOT_CONVERGED: return "FOCK_ERR_NOT_CONVERGED";
  }
  return "FOCK_ERR_UNKNOWN";
}

fock_status fock_boys_table_info(double out[4]) {
  if (!out) return FOCK_ERR_INVALID_ARG;
  out[0] = BOYS_H;
  out[1] = BOYS_NGRID;
  out[2] = BOYS_NORD;
  out[3] = BOYS_TMAX;
  return FOCK_OK;
}

fock_status fock_boys_host(int32_t mmax, double T, double *F) {
  if (!F || mmax < 0 || mmax > LTOT || !(T >= 0.0) || !isfinite(T)) return FOCK_ERR_INVALID_ARG;
  boys_eval_host(mmax, T, F);
  return FOCK_OK;
}

int32_t fock_hermite_count(int32_t la, int32_t lb) {
  if (la < 0 || lb < 0 || la > LMAX || lb > LMAX) return -1;
  return hermite_count(la, lb);
}

fock_status fock_hermite_e(int32_t la, int32_t lb, double alpha, const double *A, double beta, const double *B,
                           double *out) {
  if (la < 0 || lb < 0 || la > LMAX || lb > LMAX || !A || !B || !out || !(alpha > 0) || !(beta > 0))
    return FOCK_ERR_INVALID_ARG;
  hermite_pair(la, lb, alpha, A, beta, B, false, out);
  return FOCK_OK;
}

int32_t fock_nbasis(const fock_shellpairs *sp) { return sp ? sp->nbf : -1; }

int32_t fock_kernels_per_build(const fock_shellpairs *sp) {
  if (!sp) return -1;
  int n = 2;  // density preparation + symmetrisation
  const bool mixed = sp->opts.precision == FOCK_MIXED && sp->opts.fp32_cutoff > 0.0;
  for (const Tier &t : sp->tiers)
    if (t.nunits > 0) n += (mixed && t.reg_cb < 0) ? 2 : 1;  // group tiers: FP64 and FP32 parts
  return n;
}

extern "C++" {
namespace fk {
fock_opts default_opts() {
  fock_opts o{};
  o.precision = FOCK_FP64;
  o.fp32_cutoff = 1e-5;
  o.prune_eps = 1e-3;
  o.k_mode = FOCK_K_EXACT;
  o.k_thresh = 5e-6;
  return o;
}

bool valid_opts(const fock_opts &o) {
  if (o.precision != FOCK_FP64 && o.precision != FOCK_MIXED) return false;
  if (!(o.prune_eps >= 0.0) || o.group_override < 0 || o.group_override > 32 || o.warp_scratch < 0 ||
      (o.group_override & (o.group_override - 1)) != 0)
    return false;
  if (o.tune_isolate != 0 && o.tune_isolate != 1) return false;
  if (o.k_mode != FOCK_K_EXACT && o.k_mode != FOCK_K_DECAY_BOUND) return false;
  if (o.k_mode == FOCK_K_DECAY_BOUND && !(o.k_thresh > 0.0 && isfinite(o.k_thresh))) return false;
  for (int i = 0; i < FOCK_NCLASS * FOCK_NCLASS; ++i) {
    const int v = o.schedule[i];
    if (!(v == -1 || v == 0 || v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32)) return false;
  }
  return true;
}
}  // namespace fk
}  // extern "C++"

int32_t fock_opts_size(void) { return (int32_t)sizeof(fock_opts); }

fock_status fock_shellpairs_free(fock_shellpairs *sp) {
  if (!sp) return FOCK_OK;
  if (sp->d_block) cudaFree(sp->d_block);
  delete sp;
  return FOCK_OK;
}

fock_status fock_shellpairs_build(const fock_basis_desc *desc, const fock_opts *opts, double schwarz_thresh,
                                  cudaStream_t stream, fock_shellpairs **out) {
  if (!out) return FOCK_ERR_INVALID_ARG;
  *out = nullptr;
  fock_status vs = validate(desc);
  if (vs != FOCK_OK) return vs;
  if (!(schwarz_thresh > 0.0) || !isfinite(schwarz_thresh)) return FOCK_ERR_INVALID_ARG;
  const fock_opts o = opts ? *opts : default_opts();
  if (!valid_opts(o)) return FOCK_ERR_INVALID_ARG;

  cudaError_t ce = upload_tables(stream);
  if (ce != cudaSuccess) return to_status(ce);
  const ClassTables &ct = class_tables();

  fock_shellpairs *sp = new (std::nothrow) fock_shellpairs();
  if (!sp) return FOCK_ERR_OOM;
  cudaGetDevice(&sp->device);
  sp->opts = o;
  sp->tau_build = schwarz_thresh;
  sp->prune_eps = o.prune_eps;
  const int ns = desc->nshell;
  sp->nshell = ns;

  // ---- shells --------------------------------------------------------------
  Staging st;
  st.sxyz.assign(desc->center, desc->center + 3 * ns);
  st.shl.resize(6 * ns);
  for (int s = 0; s < ns; ++s)
    for (int x = 0; x < 3; ++x) {
      const double c = desc->center[3 * s + x];
      const float hi = (float)c;
      st.shl[6 * s + x] = hi;
      st.shl[6 * s + 3 + x] = (float)(c - (double)hi);
    }
  st.sl.assign(desc->l, desc->l + ns);
  st.sbf.resize(ns);
  int nbf = 0;
  for (int s = 0; s < ns; ++s) {
    st.sbf[s] = nbf;
    nbf += ncart(desc->l[s]);
  }
  sp->nbf = nbf;
  std::vector<std::vector<double>> cn(ns);
  for (int s = 0; s < ns; ++s) {
    cn[s].resize(desc->nprim[s]);
    norm_coefs(desc, s, cn[s].data());
  }

  // ---- all canonical pairs with all primitive pairs -------------------------
  Staging all = st;
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b) {
      const int la = desc->l[a], lb = desc->l[b];
      if (!(la > lb || (la == lb && a >= b))) continue;
      const double *A = desc->center + 3 * a, *B = desc->center + 3 * b;
      const double AB2 = (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]);
      const int Ka = desc->nprim[a], Kb = desc->nprim[b];
      const int first = (int)all.pz.size();
      for (int i = 0; i < Ka; ++i)
        for (int j = 0; j < Kb; ++j) {
          const double al = desc->exps[desc->prim_off[a] + i], be = desc->exps[desc->prim_off[b] + j];
          const double p = al + be;
          const PZ pz{(al * A[0] + be * B[0]) / p, (al * A[1] + be * B[1]) / p, (al * A[2] + be * B[2]) / p, p};
          all.pz.push_back(pz);
          all.pf.push_back(make_float4((float)pz.x, (float)pz.y, (float)pz.z, (float)p));
          all.paf.push_back(make_float4((float)(pz.x - A[0]), (float)(pz.y - A[1]), (float)(pz.z - A[2]), (float)p));
          // U_P sqrt(zeta) (2/sqrt(pi))^(1/2), so that U_P U_Q 2 sqrt(alpha/pi) = Us_P Us_Q / sqrt(zeta + eta)
          all.U.push_back(cn[a][i] * cn[b][j] * pow(kPi / p, 1.5) * exp(-al * be / p * AB2) * sqrt(p) *
                          sqrt(2.0 / sqrt(kPi)));
          all.eoff.push_back((int)all.E.size());
          const size_t e0 = all.E.size();
          const int ne = ct.nE[pair_class(la, lb)];
          all.E.resize(e0 + ne);
          hermite_pair(la, lb, al, A, be, B, true, all.E.data() + e0);
          // the pair factor Us_P is folded into the pair's Hermite coefficients, so
          // that a primitive quartet's seed prefactor is 1/sqrt(zeta + eta) alone
          for (int k = 0; k < ne; ++k) all.E[e0 + k] *= all.U.back();
        }
      all.ab.push_back(make_int2(a, b));
      all.prim.push_back(make_int2(first, Ka * Kb));
      all.cls.push_back(pair_class(la, lb));
      all.G.push_back(0.0);
    }
  const int npair_all = (int)all.ab.size();
  const int nprim_all = (int)all.pz.size();

  // ---- Schwarz factors on the GPU ------------------------------------------
  std::vector<double> Gpair(npair_all), Gprim(nprim_all);
  {
    void *base = nullptr;
    DevPairs dp{};
    std::vector<Unit> none;
    fock_status s = upload(all, none, &base, dp, nullptr, nullptr, stream);
    if (s != FOCK_OK) {
      delete sp;
      return s;
    }
    dp.nshell = ns;
    dp.nbf = nbf;
    double *dG = nullptr;
    ce = cudaMalloc(&dG, sizeof(double) * (npair_all + nprim_all + 1));
    if (ce == cudaSuccess) ce = launch_schwarz(dp, dG, dG + npair_all, stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(Gpair.data(), dG, sizeof(double) * npair_all, cudaMemcpyDeviceToHost, stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(Gprim.data(), dG + npair_all, sizeof(double) * nprim_all, cudaMemcpyDeviceToHost, stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
    if (dG) cudaFree(dG);
    cudaFree(base);
    if (ce != cudaSuccess) {
      delete sp;
      return to_status(ce, "Schwarz kernel");
    }
  }

  // ---- pruning (Sec. 3.2 primitive screening) -------------------------------
  double gmax = 0.0;
  for (double g : Gpair) gmax = std::max(gmax, g);
  const double tau = schwarz_thresh;
  struct PairRec {
    int idx, cls, nkeep, bucket;
    double G;
  };
  std::vector<PairRec> keep;
  std::vector<std::vector<int>> kept_prims(npair_all);
  for (int P = 0; P < npair_all; ++P) {
    if (Gpair[P] * gmax < tau) continue;
    const int2 pr = all.prim[P];
    for (int i = pr.x; i < pr.x + pr.y; ++i)
      if (!(o.prune_eps > 0.0 && Gprim[i] * gmax < tau * o.prune_eps)) kept_prims[P].push_back(i);
    if (kept_prims[P].empty()) continue;
    // strongest primitive pairs first, so that the primitive-quartet test can
    // end a primitive loop at its first skip (Sec. 3.2 ordering by G_[ab])
    std::stable_sort(kept_prims[P].begin(), kept_prims[P].end(),
                     [&Gprim](int x, int y) { return Gprim[x] > Gprim[y]; });
    const int nk = (int)kept_prims[P].size();
    keep.push_back({P, all.cls[P], nk, bucket_of(nk), Gpair[P]});
  }
  std::stable_sort(keep.begin(), keep.end(), [](const PairRec &x, const PairRec &y) {
    if (x.cls != y.cls) return x.cls < y.cls;
    if (x.bucket != y.bucket) return x.bucket < y.bucket;
    return x.G > y.G;
  });
  const int npair = (int)keep.size();
  // ---- decay-bound radii (Sec. 4.3.1): R_s the largest centre distance from
  // shell s to a shell it forms a kept pair with (the paper's condition on
  // G_[ac] read as "significant"), G_s the largest Schwarz factor of those
  // pairs; atoms from the description, else shells sharing a centre -------
  {
    sp->h_R.assign(ns, 0.0);
    sp->h_Gs.assign(ns, 0.0);
    for (const PairRec &r : keep) {
      const int a = all.ab[r.idx].x, b = all.ab[r.idx].y;
      double d2 = 0.0;
      for (int x = 0; x < 3; ++x) {
        const double t = desc->center[3 * a + x] - desc->center[3 * b + x];
        d2 += t * t;
      }
      const double d = sqrt(d2);
      sp->h_R[a] = std::max(sp->h_R[a], d);
      sp->h_R[b] = std::max(sp->h_R[b], d);
      sp->h_Gs[a] = std::max(sp->h_Gs[a], r.G);
      sp->h_Gs[b] = std::max(sp->h_Gs[b], r.G);
    }
    st.satom.resize(ns);
    for (int s = 0; s < ns; ++s) {
      if (desc->atom) {
        st.satom[s] = desc->atom[s];
        continue;
      }
      st.satom[s] = s;
      for (int t = 0; t < s; ++t)
        if (desc->center[3 * t] == desc->center[3 * s] && desc->center[3 * t + 1] == desc->center[3 * s + 1] &&
            desc->center[3 * t + 2] == desc->center[3 * s + 2]) {
          st.satom[s] = st.satom[t];
          break;
        }
    }
    if (o.k_mode == FOCK_K_DECAY_BOUND) {  // GDG factors n_z G_xz of kept pairs (both orders)
      st.Gn.assign((size_t)ns * ns, 0.0f);
      for (const PairRec &r : keep) {
        const int a = all.ab[r.idx].x, b = all.ab[r.idx].y;
        st.Gn[(size_t)a * ns + b] = (float)(r.G * ncart(desc->l[b]));
        st.Gn[(size_t)b * ns + a] = (float)(r.G * ncart(desc->l[a]));
      }
    }
    st.sRG.resize(ns);
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int s = 0; s < ns; ++s) {
      st.sRG[s] = make_float2((float)sp->h_R[s], (float)sp->h_Gs[s]);
      for (int x = 0; x < 3; ++x) {
        lo[x] = std::min(lo[x], desc->center[3 * s + x]);
        hi[x] = std::max(hi[x], desc->center[3 * s + x]);
      }
    }
    double diag2 = 0.0;
    for (int x = 0; x < 3; ++x) diag2 += (hi[x] - lo[x]) * (hi[x] - lo[x]);
    sp->decay_nbins = (int)floor(sqrt(diag2) / 0.5) + 2;
  }
  for (const PairRec &r : keep) {
    const int P = r.idx;
    st.ab.push_back(all.ab[P]);
    st.G.push_back(Gpair[P]);
    st.Gf.push_back((float)Gpair[P]);
    st.cls.push_back(all.cls[P]);
    st.prim.push_back(make_int2((int)st.pz.size(), r.nkeep));
    for (int i : kept_prims[P]) {
      st.pz.push_back(all.pz[i]);
      st.pf.push_back(all.pf[i]);
      st.paf.push_back(all.paf[i]);
      st.U.push_back(all.U[i]);
      st.Uf.push_back((float)all.U[i]);
      st.Gp.push_back(Gprim[i]);
      st.Gpf.push_back((float)Gprim[i]);
      st.eoff.push_back((int)st.E.size());
      const int n = ct.nE[all.cls[P]];
      st.E.insert(st.E.end(), all.E.begin() + all.eoff[i], all.E.begin() + all.eoff[i] + n);
      for (int k = 0; k < n; ++k) st.Ef.push_back((float)all.E[all.eoff[i] + k]);
    }
  }

  // ---- bins and work units --------------------------------------------------
  struct Bin {
    int begin, end, cls, bucket, nprim;  // nprim: largest kept primitive-pair count
  };
  std::vector<Bin> bins;
  for (int i = 0; i < npair; ++i) {
    if (bins.empty() || bins.back().cls != keep[i].cls || bins.back().bucket != keep[i].bucket)
      bins.push_back({i, i, keep[i].cls, keep[i].bucket, 0});
    bins.back().end = i + 1;
    bins.back().nprim = std::max(bins.back().nprim, keep[i].nkeep);
  }
  struct Task {
    int bra, ket;  // bin indices
    bool same;
    double cost;   // per quartet estimate
    int G, scratch;
    bool reg;      // served by a per-class register kernel
    int tag;       // class pair + 1 when every class pair is launched apart
  };
  std::vector<Task> tasks;
  for (int x = 0; x < (int)bins.size(); ++x)
    for (int y = x; y < (int)bins.size(); ++y) {
      const Bin &X = bins[x], &Y = bins[y];
      int lxa, lxb, lya, lyb;
      class_l(X.cls, lxa, lxb);
      class_l(Y.cls, lya, lyb);
      const double px = X.nprim, py = Y.nprim;
      const int Lx = lxa + lxb, Ly = lya + lyb, nx = ncart(lxa) * ncart(lxb), ny = ncart(lya) * ncart(lyb);
      // cost with X as bra vs Y as bra
      const double cxy = px * (py * flops_prim(Lx, Lx + Ly, Y.cls) + flops_bra(X.cls, ny));
      const double cyx = py * (px * flops_prim(Ly, Lx + Ly, X.cls) + flops_bra(Y.cls, nx));
      Task t;
      t.same = (x == y);
      if (t.same || cxy <= cyx) {
        t.bra = x;
        t.ket = y;
        t.cost = cxy;
      } else {
        t.bra = y;
        t.ket = x;
        t.cost = cyx;
      }
      int la, lb, lc, ld;
      class_l(bins[t.bra].cls, la, lb);
      class_l(bins[t.ket].cls, lc, ld);
      t.scratch = scratch_doubles(la, lb, lc, ld);
      const int c1 = std::min(X.cls, Y.cls), c2 = std::max(X.cls, Y.cls);
      const int sched = o.group_override > 0 ? 0 : o.schedule[c1 * FOCK_NCLASS + c2];
      t.tag = o.tune_isolate ? c1 * FOCK_NCLASS + c2 + 1 : 0;
      const int budget = o.warp_scratch > 0 ? o.warp_scratch : 1536;
      int G = 1;
      while (G < 32 && (32 / G) * t.scratch > budget) G *= 2;
      const int forced = o.group_override > 0 ? o.group_override : (sched > 0 ? sched : 0);
      if (forced > 0) {  // forced group size, raised where one warp's scratch would not fit
        G = forced;
        while (G < 32 && (32 / G) * t.scratch > 24000) G *= 2;
      }
      t.G = G;
      {
        const int reg_max = o.reg_max_L == 0 ? 4 : o.reg_max_L;
        const int Ltot = lxa + lxb + lya + lyb;
        const bool avail = reg_class_pair(bins[t.bra].cls, bins[t.ket].cls);
        if (sched == -1)
          t.reg = avail;
        else if (sched > 0)
          t.reg = false;
        else
          t.reg = o.group_override == 0 && Ltot <= reg_max && avail;
      }
      // mixed precision: the FP32 quartets of a total-L = 5 class pair run on
      // its FP32 register kernel (k_reg32), so the pair gets group tiers of
      // its own (its FP64 quartets stay on the group kernel)
      if (!t.reg && !o.tune_isolate && o.group_override == 0 && o.precision == FOCK_MIXED && o.fp32_cutoff > 0.0 &&
          reg32_available(bins[t.bra].cls, bins[t.ket].cls))
        t.tag = kReg32Tag + bins[t.bra].cls * FOCK_NCLASS + bins[t.ket].cls;
      tasks.push_back(t);
    }
  std::stable_sort(tasks.begin(), tasks.end(), [](const Task &a, const Task &b) { return a.cost > b.cost; });

  // tiers keyed by (G, scratch bucket)
  struct TierKey {
    int G, sb, cb, ck;  // cb >= 0: register kernel of (bra class, ket class)
    int tag;
    bool operator<(const TierKey &o2) const {
      if (tag != o2.tag) return tag < o2.tag;
      if (cb != o2.cb) return cb < o2.cb;
      if (ck != o2.ck) return ck < o2.ck;
      return G != o2.G ? G < o2.G : sb < o2.sb;
    }
    bool operator==(const TierKey &o2) const {
      return G == o2.G && sb == o2.sb && cb == o2.cb && ck == o2.ck && tag == o2.tag;
    }
  };
  auto key_of = [&bins](const Task &t) {
    if (t.reg) return TierKey{1, 0, bins[t.bra].cls, bins[t.ket].cls, t.tag};
    int sb = 0;
    while ((1 << sb) < t.scratch) ++sb;
    if (t.G < 32) sb = 0;  // one tier per G below a full warp
    return TierKey{t.G, sb, -1, -1, t.tag};
  };
  std::vector<TierKey> keys;
  for (const Task &t : tasks) {
    TierKey k = key_of(t);
    if (std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
  }
  std::sort(keys.begin(), keys.end());
  std::vector<Unit> all_units;
  std::vector<int> unit_tier;
  for (size_t ki = 0; ki < keys.size(); ++ki) {
    Tier tier{};
    tier.G = keys[ki].G;
    tier.reg_cb = keys[ki].cb;
    tier.reg_ck = keys[ki].ck;
    tier.sb = keys[ki].sb;
    tier.tag = keys[ki].tag;
    tier.mixed = (o.precision == FOCK_MIXED && o.fp32_cutoff > 0.0) ? 1 : 0;
    if (tier.tag >= kReg32Tag) {
      tier.r32_cb = (tier.tag - kReg32Tag) / FOCK_NCLASS;
      tier.r32_ck = (tier.tag - kReg32Tag) % FOCK_NCLASS;
    }
    int stride = 1;
    const int chunk = (32 / tier.G) * 8;
    const size_t first = all_units.size();
    for (const Task &t : tasks) {
      if (!(key_of(t) == keys[ki])) continue;
      stride = std::max(stride, t.scratch);
      const Bin &B = bins[t.bra], &K = bins[t.ket];
      for (int i = B.begin; i < B.end; ++i) {
        const double gi = st.G[i];
        const int k0 = t.same ? i : K.begin;
        // kets sorted by G descending: last index with G_i G_j >= tau
        int lo = k0, hi = K.end;
        while (lo < hi) {
          const int mid = (lo + hi) / 2;
          if (gi * st.G[mid] >= tau)
            lo = mid + 1;
          else
            hi = mid;
        }
        for (int j = k0; j < lo; j += chunk) all_units.push_back(Unit{i, j, std::min(lo, j + chunk), 0});
      }
    }
    if (stride % 2 == 0) ++stride;
    tier.stride = stride;
    tier.nunits = (int)(all_units.size() - first);
    sp->tiers.push_back(tier);
    for (size_t u = first; u < all_units.size(); ++u) unit_tier.push_back((int)ki);
  }

  // ---- upload compact data --------------------------------------------------
  Unit *d_units = nullptr;
  fock_status s = upload(st, all_units, &sp->d_block, sp->dev, &d_units, &sp->bytes, stream);
  if (s != FOCK_OK) {
    delete sp;
    return s;
  }
  sp->dev.nshell = ns;
  sp->dev.nbf = nbf;
  size_t uoff = 0;
  for (Tier &t : sp->tiers) {
    t.d_units = d_units + uoff;
    uoff += t.nunits;
    ce = configure_tier(t);
    if (ce != cudaSuccess) {
      fock_shellpairs_free(sp);
      return to_status(ce, "configure_tier");
    }
  }
  ce = cudaStreamSynchronize(stream);
  if (ce != cudaSuccess) {
    fock_shellpairs_free(sp);
    return to_status(ce);
  }
  sp->h_sxyz = st.sxyz;
  sp->h_sbf = st.sbf;
  sp->h_sl = st.sl;
  sp->h_ab = st.ab;
  sp->h_G = st.G;
  sp->h_prim = st.prim;
  sp->h_cls = st.cls;
  sp->h_units = std::move(all_units);
  sp->h_unit_tier = std::move(unit_tier);
  sp->host = std::move(st);
  static std::atomic<unsigned long long> next_serial{1};
  sp->serial = next_serial++;
  *out = sp;
  return FOCK_OK;
}

extern "C++" {
namespace fk {
ScratchLayout scratch_layout(const fock_shellpairs *sp) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t ns = sp->nshell, n = sp->nbf, nt = sp->tiers.size();
  const bool mixed = sp->opts.precision == FOCK_MIXED && sp->opts.fp32_cutoff > 0.0;
  const bool decay = sp->opts.k_mode == FOCK_K_DECAY_BOUND;
  ScratchLayout L;
  L.cnt_off = al(sizeof(double) * ns * ns);
  L.df_off = al(L.cnt_off + sizeof(int) * (2 * nt + 1));
  L.dshf_off = mixed ? al(L.df_off + sizeof(float) * n * n) : L.df_off;
  L.total = L.dshf_off + sizeof(float) * ns * ns;
  if (decay) {
    L.w_off = al(L.total);
    L.bins_off = al(L.w_off + sizeof(float) * ns * ns);
    L.hl_off = al(L.bins_off + sizeof(double) * sp->decay_nbins);
    L.t_off = al(L.hl_off + 2 * sizeof(double));
    L.gdg_off = al(L.t_off + sizeof(float) * ns * ns);
    L.total = L.gdg_off + sizeof(float) * ns * ns;
  }
  return L;
}

// fock_build_jk with, when ev is given (tiers + 1 events), an event recorded
// before every tier launch and one after the last.
fock_status build_jk_events(const fock_shellpairs *sp, const double *D, double schwarz_thresh, double *J,
                            double *K, cudaStream_t stream, const cudaEvent_t *ev) {
  if (!sp || !D || (!J && !K)) return FOCK_ERR_INVALID_ARG;
  if (!(schwarz_thresh >= sp->tau_build) || !isfinite(schwarz_thresh)) return FOCK_ERR_INVALID_ARG;
  const int ns = sp->nshell, n = sp->nbf;
  const size_t nt = sp->tiers.size();
  const bool mixed = sp->opts.precision == FOCK_MIXED && sp->opts.fp32_cutoff > 0.0;
  const ScratchLayout L = scratch_layout(sp);
  char *scratch = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&scratch, L.total, stream);
  if (e != cudaSuccess) return to_status(e);
  double *Dsh = (double *)scratch;
  int *counters = (int *)(scratch + L.cnt_off);
  float *Df = mixed ? (float *)(scratch + L.df_off) : nullptr;
  float *Dshf = (float *)(scratch + L.dshf_off);
  CallParts cp;
  cp.parts = (J ? 1 : 0) | (K ? 2 : 0);
  const bool decay = sp->opts.k_mode == FOCK_K_DECAY_BOUND && K;
  const bool chk = sync_check();
  const char *where = "memset";
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
  static char tier_name[64];
  for (size_t t = 0; t < nt && e == cudaSuccess; ++t) {
    snprintf(tier_name, sizeof(tier_name), "k_jk tier %zu (G=%d, smem=%zu)", t, sp->tiers[t].G, sp->tiers[t].smem);
    where = tier_name;
    if (ev) e = cudaEventRecord(ev[t], stream);
    if (e == cudaSuccess)
      e = launch_jk_tier(sp->tiers[t], sp->dev, D, Dsh, schwarz_thresh, sp->prune_eps, J, K, counters + t,
                         counters + nt + t, stream, Df, sp->opts.fp32_cutoff, Dshf, cp);
    if (e == cudaSuccess && chk) e = cudaStreamSynchronize(stream);
  }
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[nt], stream);
  if (e == cudaSuccess) {
    where = "k_symmetrize";
    e = launch_symmetrize(J, K, n, stream);
    if (e == cudaSuccess && chk) e = cudaStreamSynchronize(stream);
  }
  cudaError_t e2 = cudaFreeAsync(scratch, stream);
  if (e == cudaSuccess) {
    e = e2;
    where = "cudaFreeAsync";
  }
  return to_status(e, where);
}
}  // namespace fk
}  // extern "C++"

fock_status fock_build_jk(const fock_shellpairs *sp, const double *D, double schwarz_thresh, double *J, double *K,
                          cudaStream_t stream) {
  return build_jk_events(sp, D, schwarz_thresh, J, K, stream, nullptr);
}

fock_status fock_stream_status(cudaStream_t stream) {
  int v = 0;
  int rc = read_and_clear_status(stream, &v);
  if (rc) return FOCK_ERR_CUDA;
  return (fock_status)v;
}

fock_status fock_decay_bound(const fock_shellpairs *sp, const double *D, double out_HL[2], double *R, double *G,
                             cudaStream_t stream) {
  if (!sp || !D || !out_HL) return FOCK_ERR_INVALID_ARG;
  const int ns = sp->nshell;
  const size_t bins_off = (sizeof(double) * (size_t)ns * ns + 255) & ~(size_t)255;
  const size_t hl_off = (bins_off + sizeof(double) * sp->decay_nbins + 255) & ~(size_t)255;
  char *scratch = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&scratch, hl_off + 2 * sizeof(double), stream);
  if (e != cudaSuccess) return to_status(e, "cudaMallocAsync");
  const char *where = "k_dprep";
  e = launch_dprep(D, sp->nbf, sp->dev.sbf, sp->dev.sl, ns, (double *)scratch, stream);
  if (e == cudaSuccess) {
    where = "decay bound";
    e = launch_decay_bound(sp->dev, (double *)scratch, sp->decay_nbins, (double *)(scratch + bins_off),
                           (double *)(scratch + hl_off), nullptr, stream);
  }
  if (e == cudaSuccess) {
    where = "copy";
    e = cudaMemcpyAsync(out_HL, scratch + hl_off, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream);
  }
  cudaError_t e2 = cudaFreeAsync(scratch, stream);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return to_status(e, where);
  for (int s = 0; s < ns; ++s) {
    if (R) R[s] = sp->h_R[s];
    if (G) G[s] = sp->h_Gs[s];
  }
  return FOCK_OK;
}

fock_status fock_work_stats(const fock_shellpairs *sp, const double *D_host, double schwarz_thresh, double out[10]) {
  if (!sp || !D_host || !out) return FOCK_ERR_INVALID_ARG;
  if (!(schwarz_thresh >= sp->tau_build)) return FOCK_ERR_INVALID_ARG;
  const int ns = sp->nshell, n = sp->nbf;
  std::vector<double> Dsh((size_t)ns * ns, 0.0);
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b) {
      double mx = 0.0;
      for (int i = 0; i < ncart(sp->h_sl[a]); ++i)
        for (int j = 0; j < ncart(sp->h_sl[b]); ++j)
          mx = std::max(mx, fabs(D_host[(size_t)(sp->h_sbf[a] + i) * n + sp->h_sbf[b] + j]));
      Dsh[(size_t)a * ns + b] = mx;
    }
  const double tau = schwarz_thresh;
  const bool mixed = sp->opts.precision == FOCK_MIXED && sp->opts.fp32_cutoff > 0.0;
  const double *Gp = sp->host.Gp.data();
  const double teps = sp->prune_eps > 0.0 ? tau * sp->prune_eps : 0.0;
  const FlopTable &ft = flop_table();
  // acc: quartets / ERIs passing Schwarz, evaluated quartets / ERIs, primitive
  // quartets, modelled flops, FP32 quartets, FP32 flops
  auto count_units = [&](size_t u0, size_t u1, double *acc) {
    for (size_t ui = u0; ui < u1; ++ui) {
      const Unit &u = sp->h_units[ui];
      const int P = u.bra;
      const int2 ab = sp->h_ab[P];
      // the register kernels also run the primitive quartets of an FP64
      // quartet that lie below the cutoff in FP32; the group kernels do not
      const bool reg_tier = sp->tiers[sp->h_unit_tier[ui]].reg_cb >= 0;
      for (int Q = u.k0; Q < u.k1; ++Q) {
        const int2 cd = sp->h_ab[Q];
        const double g = sp->h_G[P] * sp->h_G[Q];
        if (g < tau) continue;
        const int la = sp->h_sl[ab.x], lb = sp->h_sl[ab.y], lc = sp->h_sl[cd.x], ld = sp->h_sl[cd.y];
        const double ne = (double)ncart(la) * ncart(lb) * ncart(lc) * ncart(ld);
        acc[0] += 1;
        acc[1] += ne;
        double dm = Dsh[(size_t)ab.x * ns + ab.y];
        dm = std::max(dm, Dsh[(size_t)cd.x * ns + cd.y]);
        dm = std::max(dm, Dsh[(size_t)ab.x * ns + cd.x]);
        dm = std::max(dm, Dsh[(size_t)ab.x * ns + cd.y]);
        dm = std::max(dm, Dsh[(size_t)ab.y * ns + cd.x]);
        dm = std::max(dm, Dsh[(size_t)ab.y * ns + cd.y]);
        if (g * dm < tau) continue;
        acc[2] += 1;
        acc[3] += ne;
        // primitive quartets the kernels evaluate (same skip rule and order)
        const int2 pb = sp->h_prim[P], pk = sp->h_prim[Q];
        const bool split = mixed && reg_tier && !(g * dm < sp->opts.fp32_cutoff);
        double np = 0.0, nbra = 0.0, np32 = 0.0, nbra32 = 0.0, nbra64 = 0.0;
        for (int ip = pb.x; ip < pb.x + pb.y; ++ip) {
          int n = 0, n32 = 0;
          for (int jq = pk.x; jq < pk.x + pk.y; ++jq) {
            const double x = Gp[ip] * Gp[jq] * dm;
            if (x < teps) break;
            ++n;
            if (split && x < sp->opts.fp32_cutoff) ++n32;
          }
          if (n == 0) break;
          np += n;
          nbra += 1;
          np32 += n32;
          if (n32 > 0) nbra32 += 1;
          if (n > n32) nbra64 += 1;
        }
        acc[4] += np;
        const double fp = ft.prim[sp->h_cls[P]][sp->h_cls[Q]], fb = ft.bra[sp->h_cls[P]][sp->h_cls[Q]];
        if (mixed && g * dm < sp->opts.fp32_cutoff) {
          const double f = np * fp + nbra * fb + 12.0 * ne;
          acc[5] += f;
          acc[6] += 1;
          acc[7] += f;
        } else {
          const double f32 = np32 * fp + nbra32 * fb;
          acc[5] += (np - np32) * fp + nbra64 * fb + 12.0 * ne + f32;
          acc[7] += f32;
        }
      }
    }
  };
  // every count is an integer below 2^53, so the per-thread partial sums add
  // up exactly whatever the split
  const size_t nu = sp->h_units.size();
  const unsigned hw = std::thread::hardware_concurrency();
  const int nthr = (int)std::max<size_t>(1, std::min<size_t>({(size_t)(hw ? hw : 1), (size_t)32, nu / 64 + 1}));
  std::vector<std::array<double, 8>> part(nthr);
  for (auto &a : part) a.fill(0.0);
  {
    std::vector<std::thread> pool;
    for (int t = 0; t < nthr; ++t)
      pool.emplace_back([&, t] { count_units(nu * t / nthr, nu * (t + 1) / nthr, part[t].data()); });
    for (auto &th : pool) th.join();
  }
  double tot[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (const auto &a : part)
    for (int k = 0; k < 8; ++k) tot[k] += a[k];
  const double q1 = tot[0], e1 = tot[1], q2 = tot[2], e2 = tot[3], pq = tot[4], fl = tot[5], q32 = tot[6],
               fl32 = tot[7];
  double nprim = 0;
  for (const int2 &p : sp->h_prim) nprim += p.y;
  out[0] = q1;
  out[1] = e1;
  out[2] = q2;
  out[3] = e2;
  out[4] = pq;
  out[5] = fl;
  out[6] = nprim;
  out[7] = (double)sp->h_ab.size();
  out[8] = q32;
  out[9] = fl32;
  return FOCK_OK;
}

}  // extern "C"
