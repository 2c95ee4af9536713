/*
 * CPU reference ("oracle") for the Coulomb (J) and exchange (K) build of
 * arXiv:2407.21445. TEST INFRASTRUCTURE ONLY: it is linked by the test suite,
 * by the smoke check and by the benchmark's CPU-baseline leg, never by the
 * GPU library. It shares no code, table or header with the GPU path.
 *
 * What it computes (all FP64, plain loops, OpenMP over shell quartets):
 *   - contracted Cartesian Gaussian basis functions (Sec. 2.1, Eqs. cgf/prim),
 *     each Cartesian function normalised to unit self-overlap;
 *   - the Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt (Eq. boys-fn-def)
 *     by its power series plus downward recursion, or by the error function
 *     plus upward recursion for large T;
 *   - primitive ERIs by the Obara-Saika / Head-Gordon-Pople vertical
 *     recurrences (Eqs. vrr1, vrr2), contraction over primitives, then the
 *     horizontal recurrences (Eq. hrr) -- deliberately a different recursion
 *     family from the McMurchie-Davidson scheme the GPU kernels use;
 *   - Schwarz factors G_ab and primitive G_[ab] (Eqs. cauchy-schwarz 1, 2);
 *   - J_mn = sum_ls (mn|ls) D_ls and K_mn = sum_ls (ml|ns) D_ls (Sec. 2.2,
 *     Eq. fock_build) with explicit 8-fold permutational scatter (Sec. 2.3).
 *
 * Readings of the paper taken here (garbled or silent passages):
 *   - the auxiliary integral is [00|00]^(m) = U_P U_Q (2 theta / sqrt(pi)) F_m(T);
 *   - in vrr2 the PQ coefficient is W-Q = +zeta/(zeta+eta) (P-Q);
 *   - screening skips a quartet iff G_ab G_cd < tau (pre-launch batch test)
 *     or G_ab G_cd Dmax < tau with Dmax the largest |D| over the six shell
 *     blocks ab, ac, ad, bc, bd, cd (in-kernel test), both Sec. 3.2;
 *   - a primitive pair is dropped iff G_[ab] * Gmax < tau * eps_p, Gmax the
 *     largest contracted G_ab (primitive-level pruning, Sec. 3.2);
 *   - inside a contracted quartet that passes, a primitive quartet [ab|cd]
 *     is skipped iff G_[ab] * G_[cd] * Dmax < tau * eps_p, Dmax the six-block
 *     maximum above (screening with the primitive Cauchy-Schwarz bound, Sec.
 *     3.2, at the level of primitive integrals as in the MMD scheme, Sec. 3.3).
 *
 * Every J/K accumulation uses Neumaier-compensated sums.
 *
 * One-electron integrals for the SCF driver (Sec. 2.2, h = T + V): overlap
 * and kinetic energy from one-dimensional Obara-Saika overlaps (kinetic as
 * 1/2 sum_x <d_x a|d_x b>), nuclear attraction by the Obara-Saika
 * nuclear-attraction vertical recurrence and the horizontal recurrence.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_LMAX 3
#define OR_EMAX (2 * OR_LMAX)       /* largest |e| in a bra/ket VRR target   */
#define OR_MMAX (4 * OR_LMAX + 1)   /* Boys orders 0..4*LMAX                 */
#define OR_NH(n) (((n) + 1) * ((n) + 2) * ((n) + 3) / 6)
#define OR_NC(l) (((l) + 1) * ((l) + 2) / 2)
#define OR_NHE OR_NH(OR_EMAX)       /* 84 Cartesian vectors with |e| <= 6    */

typedef struct {
  int nshell;
  const double *center; /* [nshell*3] bohr */
  const int32_t *l;
  const int32_t *nprim;
  const int32_t *prim_off;
  const double *exps;
  const double *coefs;
} or_basis;

/* ------------------------------------------------------------------------- */
/* Cartesian vectors: compact index over all (x,y,z) with x+y+z <= OR_EMAX,   */
/* ordered by total degree, then x descending, then y descending.             */
/* ------------------------------------------------------------------------- */
static int g_cidx[OR_EMAX + 2][OR_EMAX + 2][OR_EMAX + 2];
static int g_cvec[OR_NH(OR_EMAX + 1)][3];
static int g_tables_ready = 0;

static void or_init_tables(void) {
  if (g_tables_ready) return;
  int n = 0;
  for (int d = 0; d <= OR_EMAX + 1; ++d)
    for (int x = d; x >= 0; --x)
      for (int y = d - x; y >= 0; --y) {
        int z = d - x - y;
        g_cidx[x][y][z] = n;
        g_cvec[n][0] = x;
        g_cvec[n][1] = y;
        g_cvec[n][2] = z;
        ++n;
      }
  g_tables_ready = 1;
}

static double or_dfact(int n) { /* (n)!! for n >= -1 */
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

/* ------------------------------------------------------------------------- */
/* Boys function                                                              */
/* ------------------------------------------------------------------------- */
void oracle_boys(int mmax, double T, double *F) {
  if (T < 35.0) {
    /* F_mmax(T) = exp(-T) sum_k (2T)^k / ((2mmax+1)(2mmax+3)...(2mmax+2k+1)) */
    double term = 1.0 / (2.0 * mmax + 1.0), sum = term;
    for (int k = 1; k < 2000; ++k) {
      term *= 2.0 * T / (2.0 * mmax + 2.0 * k + 1.0);
      sum += term;
      if (term < 1e-18 * sum) break;
    }
    double et = exp(-T);
    F[mmax] = et * sum;
    for (int m = mmax - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + et) / (2.0 * m + 1.0);
  } else {
    double et = exp(-T);
    F[0] = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
    for (int m = 0; m < mmax; ++m) F[m + 1] = ((2.0 * m + 1.0) * F[m] - et) / (2.0 * T);
  }
}

/* ------------------------------------------------------------------------- */
/* normalisation                                                              */
/* ------------------------------------------------------------------------- */
/* Contraction coefficients including the primitive normalisation
 * (2a/pi)^(3/4) (4a)^(l/2) and the contracted normalisation of the shell; the
 * Cartesian factor 1/sqrt(prod (2k-1)!!) is applied per component later. */
static void or_shell_coefs(const or_basis *B, int s, double *out) {
  int l = B->l[s], K = B->nprim[s], o = B->prim_off[s];
  double S = 0.0;
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) {
      double ai = B->exps[o + i], aj = B->exps[o + j];
      S += B->coefs[o + i] * B->coefs[o + j] * pow(2.0 * sqrt(ai * aj) / (ai + aj), l + 1.5);
    }
  double nc = 1.0 / sqrt(S);
  for (int i = 0; i < K; ++i) {
    double a = B->exps[o + i];
    out[i] = nc * B->coefs[o + i] * pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * l);
  }
}

static double or_cart_norm(int x, int y, int z) {
  return 1.0 / sqrt(or_dfact(2 * x - 1) * or_dfact(2 * y - 1) * or_dfact(2 * z - 1));
}

/* ------------------------------------------------------------------------- */
/* primitive/contracted ERIs by OS/HGP                                         */
/* ------------------------------------------------------------------------- */
typedef struct {
  double *vrr;   /* [OR_NHE][OR_NHE][OR_MMAX] */
  double *cont;  /* [OR_NHE][OR_NHE] contracted (e0|f0) */
  double *h1;    /* HRR work */
  double *h2;
} or_work;

static void or_work_alloc(or_work *w) {
  w->vrr = (double *)malloc(sizeof(double) * OR_NHE * OR_NHE * OR_MMAX);
  w->cont = (double *)malloc(sizeof(double) * OR_NHE * OR_NHE);
  w->h1 = (double *)malloc(sizeof(double) * OR_NHE * OR_NHE * OR_NH(OR_LMAX));
  w->h2 = (double *)malloc(sizeof(double) * OR_NHE * OR_NH(OR_LMAX) * OR_NC(OR_LMAX) * OR_NC(OR_LMAX));
}
static void or_work_free(or_work *w) {
  free(w->vrr);
  free(w->cont);
  free(w->h1);
  free(w->h2);
}

#define VRR(e, f, m) w->vrr[((size_t)(e) * OR_NHE + (f)) * OR_MMAX + (m)]

/* Adds sum over one primitive quartet of [e0|f0]^(0) (|e|<=emax, |f|<=fmax)
 * to w->cont.  Gaussians: exponents a,b on centres A,B (bra) and c,d on C,D
 * (ket); `scale` multiplies the auxiliary integrals (contraction coefs). */
static void or_vrr_prim(or_work *w, int emax, int fmax, double a, const double *A, double b,
                        const double *Bc, double c, const double *C, double d, const double *D,
                        double scale) {
  double zeta = a + b, eta = c + d, ze = zeta + eta;
  double P[3], Q[3], PA[3], QC[3], WP[3], WQ[3], AB2 = 0.0, CD2 = 0.0, PQ2 = 0.0;
  for (int i = 0; i < 3; ++i) {
    P[i] = (a * A[i] + b * Bc[i]) / zeta;
    Q[i] = (c * C[i] + d * D[i]) / eta;
    PA[i] = P[i] - A[i];
    QC[i] = Q[i] - C[i];
    double pq = P[i] - Q[i];
    WP[i] = -eta / ze * pq;
    WQ[i] = zeta / ze * pq;
    AB2 += (A[i] - Bc[i]) * (A[i] - Bc[i]);
    CD2 += (C[i] - D[i]) * (C[i] - D[i]);
    PQ2 += pq * pq;
  }
  double rho = zeta * eta / ze;
  double UP = pow(M_PI / zeta, 1.5) * exp(-a * b / zeta * AB2);
  double UQ = pow(M_PI / eta, 1.5) * exp(-c * d / eta * CD2);
  double theta = sqrt(rho);
  int L = emax + fmax;
  double F[OR_MMAX + 1];
  oracle_boys(L, rho * PQ2, F);
  double pref = scale * UP * UQ * 2.0 * theta / sqrt(M_PI);
  for (int m = 0; m <= L; ++m) VRR(0, 0, m) = pref * F[m];
  /* vrr1: build e with f = 0 */
  for (int ie = 1; ie < OR_NH(emax); ++ie) {
    int ex = g_cvec[ie][0], ey = g_cvec[ie][1], ez = g_cvec[ie][2];
    int v[3] = {ex, ey, ez};
    int i = ex > 0 ? 0 : (ey > 0 ? 1 : 2);
    v[i] -= 1;
    int e1 = g_cidx[v[0]][v[1]][v[2]];
    int ni = v[i]; /* component of the lowered vector */
    int e2 = -1;
    if (ni > 0) {
      v[i] -= 1;
      e2 = g_cidx[v[0]][v[1]][v[2]];
    }
    int deg = ex + ey + ez;
    for (int m = 0; m <= L - deg; ++m) {
      double val = PA[i] * VRR(e1, 0, m) + WP[i] * VRR(e1, 0, m + 1);
      if (e2 >= 0) val += ni / (2.0 * zeta) * (VRR(e2, 0, m) - rho / zeta * VRR(e2, 0, m + 1));
      VRR(ie, 0, m) = val;
    }
  }
  /* vrr2: build f for every e */
  for (int jf = 1; jf < OR_NH(fmax); ++jf) {
    int fx = g_cvec[jf][0], fy = g_cvec[jf][1], fz = g_cvec[jf][2];
    int v[3] = {fx, fy, fz};
    int i = fx > 0 ? 0 : (fy > 0 ? 1 : 2);
    v[i] -= 1;
    int f1 = g_cidx[v[0]][v[1]][v[2]];
    int ni = v[i];
    int f2 = -1;
    if (ni > 0) {
      v[i] -= 1;
      f2 = g_cidx[v[0]][v[1]][v[2]];
    }
    int fdeg = fx + fy + fz;
    for (int ie = 0; ie < OR_NH(emax); ++ie) {
      int ev[3] = {g_cvec[ie][0], g_cvec[ie][1], g_cvec[ie][2]};
      int edeg = ev[0] + ev[1] + ev[2];
      int ei = ev[i];
      int em = -1;
      if (ei > 0) {
        ev[i] -= 1;
        em = g_cidx[ev[0]][ev[1]][ev[2]];
      }
      for (int m = 0; m <= L - edeg - fdeg; ++m) {
        double val = QC[i] * VRR(ie, f1, m) + WQ[i] * VRR(ie, f1, m + 1);
        if (f2 >= 0) val += ni / (2.0 * eta) * (VRR(ie, f2, m) - rho / eta * VRR(ie, f2, m + 1));
        if (em >= 0) val += ei / (2.0 * ze) * VRR(em, f1, m + 1);
        VRR(ie, jf, m) = val;
      }
    }
  }
  for (int ie = 0; ie < OR_NH(emax); ++ie)
    for (int jf = 0; jf < OR_NH(fmax); ++jf) w->cont[ie * OR_NHE + jf] += VRR(ie, jf, 0);
}

/* HRR on the ket, then on the bra (Eq. hrr), from contracted (e0|f0).
 * out[((ia*nb + ib)*nc + ic)*nd + id], Cartesian factors NOT applied. */
static void or_hrr(or_work *w, int la, int lb, int lc, int ld, const double *A, const double *Bc,
                   const double *C, const double *D, double *out) {
  int emin = la, emax = la + lb, fmin = lc, fmax = lc + ld;
  double AB[3], CD[3];
  for (int i = 0; i < 3; ++i) {
    AB[i] = A[i] - Bc[i];
    CD[i] = C[i] - D[i];
  }
  int nhd = OR_NH(ld), nhb = OR_NH(lb);
  /* h1[e][c][d]: (e0|cd), c over compact idx with |c| in [lc, fmax-|d|], d over |d|<=ld */
#define H1(e, c, d) w->h1[((size_t)(e) * OR_NHE + (c)) * nhd + (d)]
  for (int ie = OR_NH(emin - 1); ie < OR_NH(emax); ++ie)
    for (int jc = OR_NH(fmin - 1); jc < OR_NH(fmax); ++jc) H1(ie, jc, 0) = w->cont[ie * OR_NHE + jc];
  for (int jd = 1; jd < nhd; ++jd) {
    int v[3] = {g_cvec[jd][0], g_cvec[jd][1], g_cvec[jd][2]};
    int ddeg = v[0] + v[1] + v[2];
    int i = v[0] > 0 ? 0 : (v[1] > 0 ? 1 : 2);
    v[i] -= 1;
    int dm = g_cidx[v[0]][v[1]][v[2]];
    for (int jc = OR_NH(fmin - 1); jc < OR_NH(fmax - ddeg); ++jc) {
      int cv[3] = {g_cvec[jc][0], g_cvec[jc][1], g_cvec[jc][2]};
      cv[i] += 1;
      int cp = g_cidx[cv[0]][cv[1]][cv[2]];
      for (int ie = OR_NH(emin - 1); ie < OR_NH(emax); ++ie)
        H1(ie, jc, jd) = H1(ie, cp, dm) + CD[i] * H1(ie, jc, dm);
    }
  }
  /* h2[a][b][cd]: bra HRR, cd = (c,d) flattened over shell positions */
  int ncd = OR_NC(lc) * OR_NC(ld);
#define H2(a, b, cd) w->h2[((size_t)(a) * nhb + (b)) * ncd + (cd)]
  for (int ie = OR_NH(emin - 1); ie < OR_NH(emax); ++ie)
    for (int jc = OR_NH(lc - 1); jc < OR_NH(lc); ++jc)
      for (int jd = OR_NH(ld - 1); jd < OR_NH(ld); ++jd) {
        int pc = jc - OR_NH(lc - 1), pd = jd - OR_NH(ld - 1);
        H2(ie, 0, pc * OR_NC(ld) + pd) = H1(ie, jc, jd);
      }
  for (int jb = 1; jb < nhb; ++jb) {
    int v[3] = {g_cvec[jb][0], g_cvec[jb][1], g_cvec[jb][2]};
    int bdeg = v[0] + v[1] + v[2];
    int i = v[0] > 0 ? 0 : (v[1] > 0 ? 1 : 2);
    v[i] -= 1;
    int bm = g_cidx[v[0]][v[1]][v[2]];
    for (int ja = OR_NH(emin - 1); ja < OR_NH(emax - bdeg); ++ja) {
      int av[3] = {g_cvec[ja][0], g_cvec[ja][1], g_cvec[ja][2]};
      av[i] += 1;
      int ap = g_cidx[av[0]][av[1]][av[2]];
      for (int cd = 0; cd < ncd; ++cd) H2(ja, jb, cd) = H2(ap, bm, cd) + AB[i] * H2(ja, bm, cd);
    }
  }
  int nbv = OR_NC(lb);
  for (int ja = OR_NH(la - 1); ja < OR_NH(la); ++ja)
    for (int jb = OR_NH(lb - 1); jb < OR_NH(lb); ++jb)
      for (int cd = 0; cd < ncd; ++cd) {
        int pa = ja - OR_NH(la - 1), pb = jb - OR_NH(lb - 1);
        out[(pa * nbv + pb) * ncd + cd] = H2(ja, jb, cd);
      }
#undef H1
#undef H2
}

/* Primitive ERI block for unnormalised Cartesian Gaussians with unit
 * coefficients, (x-A)^a.. exp(-alpha |r-A|^2).  out: [nc(la)][nc(lb)][nc(lc)][nc(ld)]. */
int oracle_prim_eri(int la, int lb, int lc, int ld, double a, const double *A, double b,
                    const double *Bc, double c, const double *C, double d, const double *D,
                    double *out) {
  if (la < 0 || lb < 0 || lc < 0 || ld < 0 || la > OR_LMAX + 1 || lb > OR_LMAX ||
      lc > OR_LMAX || ld > OR_LMAX || la + lb > OR_EMAX || lc + ld > OR_EMAX)
    return 1;
  or_init_tables();
  or_work w;
  or_work_alloc(&w);
  memset(w.cont, 0, sizeof(double) * OR_NHE * OR_NHE);
  or_vrr_prim(&w, la + lb, lc + ld, a, A, b, Bc, c, C, d, D, 1.0);
  or_hrr(&w, la, lb, lc, ld, A, Bc, C, D, out);
  or_work_free(&w);
  return 0;
}

/* prim-pair keep mask for shell pair (s1,s2): bit i*K2+j. NULL = keep all */
typedef struct {
  const or_basis *B;
  double *coef;       /* normalised contraction coefficients, same layout as exps */
  int *bf_off;        /* first basis function of each shell */
  int nbf;
  uint64_t *keep;     /* [nshell*nshell] or NULL */
} or_ctx;

/* Contracted shell-quartet ERIs (ab|cd), normalised Cartesian functions.
 * out[((ia*nb+ib)*nc+ic)*nd+id].  Primitive pairs absent from the keep masks
 * are skipped.  Optional prim restriction (pi,pj) on the bra and ket pair for
 * primitive Schwarz factors: pass -1 to use all.
 * Primitive-quartet screening (Sec. 3.2, primitive Cauchy-Schwarz bound,
 * applied at the level of primitive integrals as the MMD scheme of Sec. 3.3
 * does): with gab, gcd the primitive factors G_[ab], G_[cd] of the two pairs
 * (indexed like the keep masks), the primitive quartet [ab|cd] is skipped
 * iff G_[ab] * G_[cd] * dm < thr.  gab == NULL: no primitive-quartet test. */
static void or_shell_quartet(const or_ctx *X, or_work *w, int sa, int sb, int sc, int sd,
                             int bra_prim, int ket_prim, const double *gab, const double *gcd, double dm,
                             double thr, double *out) {
  const or_basis *B = X->B;
  int la = B->l[sa], lb = B->l[sb], lc = B->l[sc], ld = B->l[sd];
  const double *A = B->center + 3 * sa, *Bc = B->center + 3 * sb, *C = B->center + 3 * sc,
               *D = B->center + 3 * sd;
  int Ka = B->nprim[sa], Kb = B->nprim[sb], Kc = B->nprim[sc], Kd = B->nprim[sd];
  int oa = B->prim_off[sa], ob = B->prim_off[sb], oc = B->prim_off[sc], od = B->prim_off[sd];
  uint64_t kab = X->keep ? X->keep[(size_t)sa * B->nshell + sb] : ~(uint64_t)0;
  uint64_t kcd = X->keep ? X->keep[(size_t)sc * B->nshell + sd] : ~(uint64_t)0;
  memset(w->cont, 0, sizeof(double) * OR_NHE * OR_NHE);
  for (int i = 0; i < Ka; ++i)
    for (int j = 0; j < Kb; ++j) {
      int pij = i * Kb + j;
      if (bra_prim >= 0 && pij != bra_prim) continue;
      if (!((kab >> pij) & 1)) continue;
      for (int k = 0; k < Kc; ++k)
        for (int l = 0; l < Kd; ++l) {
          int pkl = k * Kd + l;
          if (ket_prim >= 0 && pkl != ket_prim) continue;
          if (!((kcd >> pkl) & 1)) continue;
          if (gab && gab[pij] * gcd[pkl] * dm < thr) continue;
          double s = X->coef[oa + i] * X->coef[ob + j] * X->coef[oc + k] * X->coef[od + l];
          or_vrr_prim(w, la + lb, lc + ld, B->exps[oa + i], A, B->exps[ob + j], Bc,
                      B->exps[oc + k], C, B->exps[od + l], D, s);
        }
    }
  or_hrr(w, la, lb, lc, ld, A, Bc, C, D, out);
  /* Cartesian normalisation factors */
  int na = OR_NC(la), nb = OR_NC(lb), nc = OR_NC(lc), nd = OR_NC(ld);
  double fa[OR_NC(OR_LMAX)], fb[OR_NC(OR_LMAX)], fc[OR_NC(OR_LMAX)], fd[OR_NC(OR_LMAX)];
  int base;
  base = OR_NH(la - 1) * (la > 0);
  for (int i = 0; i < na; ++i) fa[i] = or_cart_norm(g_cvec[base + i][0], g_cvec[base + i][1], g_cvec[base + i][2]);
  base = OR_NH(lb - 1) * (lb > 0);
  for (int i = 0; i < nb; ++i) fb[i] = or_cart_norm(g_cvec[base + i][0], g_cvec[base + i][1], g_cvec[base + i][2]);
  base = OR_NH(lc - 1) * (lc > 0);
  for (int i = 0; i < nc; ++i) fc[i] = or_cart_norm(g_cvec[base + i][0], g_cvec[base + i][1], g_cvec[base + i][2]);
  base = OR_NH(ld - 1) * (ld > 0);
  for (int i = 0; i < nd; ++i) fd[i] = or_cart_norm(g_cvec[base + i][0], g_cvec[base + i][1], g_cvec[base + i][2]);
  for (int ia = 0; ia < na; ++ia)
    for (int ib = 0; ib < nb; ++ib)
      for (int ic = 0; ic < nc; ++ic)
        for (int id = 0; id < nd; ++id) out[((ia * nb + ib) * nc + ic) * nd + id] *= fa[ia] * fb[ib] * fc[ic] * fd[id];
}

static int or_ctx_init(or_ctx *X, const or_basis *B) {
  or_init_tables();
  X->B = B;
  int np = 0;
  X->bf_off = (int *)malloc(sizeof(int) * (B->nshell + 1));
  int n = 0;
  for (int s = 0; s < B->nshell; ++s) {
    if (B->l[s] < 0 || B->l[s] > OR_LMAX || B->nprim[s] < 1 || B->nprim[s] > 8) return 1;
    X->bf_off[s] = n;
    n += OR_NC(B->l[s]);
    int e = B->prim_off[s] + B->nprim[s];
    if (e > np) np = e;
  }
  X->bf_off[B->nshell] = n;
  X->nbf = n;
  X->coef = (double *)calloc(np > 0 ? np : 1, sizeof(double));
  for (int s = 0; s < B->nshell; ++s) or_shell_coefs(B, s, X->coef + B->prim_off[s]);
  X->keep = NULL;
  return 0;
}

static void or_ctx_free(or_ctx *X) {
  free(X->bf_off);
  free(X->coef);
  free(X->keep);
}

/* ------------------------------------------------------------------------- */
/* exported: basis helpers                                                    */
/* ------------------------------------------------------------------------- */
int oracle_nbf(int nshell, const int32_t *l) {
  int n = 0;
  for (int s = 0; s < nshell; ++s) n += OR_NC(l[s]);
  return n;
}

/* normalised contraction coefficients (Cartesian factor excluded) */
int oracle_norm_coefs(int nshell, const double *center, const int32_t *l, const int32_t *nprim,
                      const int32_t *prim_off, const double *exps, const double *coefs,
                      double *out) {
  or_basis B = {nshell, center, l, nprim, prim_off, exps, coefs};
  for (int s = 0; s < nshell; ++s) or_shell_coefs(&B, s, out + prim_off[s]);
  return 0;
}

/* Overlap matrix by the Obara-Saika overlap recursion (separate from the
 * ERI code): used to pin the normalisation (diagonal = 1). */
int oracle_overlap(int nshell, const double *center, const int32_t *l, const int32_t *nprim,
                   const int32_t *prim_off, const double *exps, const double *coefs, double *S) {
  or_basis B = {nshell, center, l, nprim, prim_off, exps, coefs};
  or_ctx X;
  if (or_ctx_init(&X, &B)) return 1;
  int N = X.nbf;
  for (int sa = 0; sa < nshell; ++sa)
    for (int sb = 0; sb < nshell; ++sb) {
      int la = l[sa], lb = l[sb];
      const double *A = center + 3 * sa, *Bc = center + 3 * sb;
      int na = OR_NC(la), nb = OR_NC(lb);
      double blk[OR_NC(OR_LMAX) * OR_NC(OR_LMAX)];
      memset(blk, 0, sizeof(blk));
      for (int i = 0; i < nprim[sa]; ++i)
        for (int j = 0; j < nprim[sb]; ++j) {
          double a = exps[prim_off[sa] + i], b = exps[prim_off[sb] + j], p = a + b;
          double s1[3][OR_LMAX + 1][OR_LMAX + 1];
          for (int x = 0; x < 3; ++x) {
            double Px = (a * A[x] + b * Bc[x]) / p;
            double XAB = A[x] - Bc[x];
            double s00 = sqrt(M_PI / p) * exp(-a * b / p * XAB * XAB);
            /* 1-D OS: S(i+1,j) = XPA S(i,j) + (i S(i-1,j) + j S(i,j-1)) / 2p */
            double t[OR_LMAX + 2][OR_LMAX + 2];
            t[0][0] = s00;
            for (int ii = 0; ii <= la; ++ii)
              for (int jj = 0; jj <= lb; ++jj) {
                if (ii == 0 && jj == 0) continue;
                double v;
                if (ii > 0) {
                  v = (Px - A[x]) * t[ii - 1][jj];
                  if (ii > 1) v += (ii - 1) * t[ii - 2][jj] / (2 * p);
                  if (jj > 0) v += jj * t[ii - 1][jj - 1] / (2 * p);
                } else {
                  v = (Px - Bc[x]) * t[ii][jj - 1];
                  if (jj > 1) v += (jj - 1) * t[ii][jj - 2] / (2 * p);
                }
                t[ii][jj] = v;
              }
            for (int ii = 0; ii <= la; ++ii)
              for (int jj = 0; jj <= lb; ++jj) s1[x][ii][jj] = t[ii][jj];
          }
          double cc = X.coef[prim_off[sa] + i] * X.coef[prim_off[sb] + j];
          int ba = OR_NH(la - 1) * (la > 0), bb = OR_NH(lb - 1) * (lb > 0);
          for (int ia = 0; ia < na; ++ia)
            for (int ib = 0; ib < nb; ++ib) {
              const int *u = g_cvec[ba + ia], *v = g_cvec[bb + ib];
              blk[ia * nb + ib] += cc * s1[0][u[0]][v[0]] * s1[1][u[1]][v[1]] * s1[2][u[2]][v[2]];
            }
        }
      int ba = OR_NH(la - 1) * (la > 0), bb = OR_NH(lb - 1) * (lb > 0);
      for (int ia = 0; ia < na; ++ia)
        for (int ib = 0; ib < nb; ++ib) {
          const int *u = g_cvec[ba + ia], *v = g_cvec[bb + ib];
          S[(size_t)(X.bf_off[sa] + ia) * N + X.bf_off[sb] + ib] =
              blk[ia * nb + ib] * or_cart_norm(u[0], u[1], u[2]) * or_cart_norm(v[0], v[1], v[2]);
        }
    }
  or_ctx_free(&X);
  return 0;
}

/* Contracted shell-quartet ERIs (no pruning), normalised functions. */
int oracle_shell_eri(int nshell, const double *center, const int32_t *l, const int32_t *nprim,
                     const int32_t *prim_off, const double *exps, const double *coefs, int sa,
                     int sb, int sc, int sd, double *out) {
  or_basis B = {nshell, center, l, nprim, prim_off, exps, coefs};
  or_ctx X;
  if (or_ctx_init(&X, &B)) return 1;
  or_work w;
  or_work_alloc(&w);
  or_shell_quartet(&X, &w, sa, sb, sc, sd, -1, -1, NULL, NULL, 0.0, 0.0, out);
  or_work_free(&w);
  or_ctx_free(&X);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Schwarz factors and pruning                                                */
/* ------------------------------------------------------------------------- */
/* G[sa*nshell+sb] = max_{mn} sqrt((mn|mn)) over the contracted pair (all
 * primitives); Gp[(sa*nshell+sb)*64 + i*Kb+j] = same for primitive pair (i,j).
 * Computed for sa >= sb and mirrored so both orders agree bit for bit. */
static void or_schwarz(const or_ctx *X, double *G, double *Gp) {
  const or_basis *B = X->B;
  int ns = B->nshell;
#pragma omp parallel
  {
    or_work w;
    or_work_alloc(&w);
    double *buf = (double *)malloc(sizeof(double) * 10000);
#pragma omp for schedule(dynamic, 1)
    for (int sa = 0; sa < ns; ++sa)
      for (int sb = 0; sb <= sa; ++sb) {
        int na = OR_NC(B->l[sa]), nb = OR_NC(B->l[sb]), nab = na * nb;
        or_shell_quartet(X, &w, sa, sb, sa, sb, -1, -1, NULL, NULL, 0.0, 0.0, buf);
        double mx = 0.0;
        for (int k = 0; k < nab; ++k) mx = fmax(mx, fabs(buf[k * nab + k]));
        G[(size_t)sa * ns + sb] = G[(size_t)sb * ns + sa] = sqrt(mx);
        int Ka = B->nprim[sa], Kb = B->nprim[sb];
        for (int i = 0; i < Ka; ++i)
          for (int j = 0; j < Kb; ++j) {
            int p = i * Kb + j;
            or_shell_quartet(X, &w, sa, sb, sa, sb, p, p, NULL, NULL, 0.0, 0.0, buf);
            double m2 = 0.0;
            for (int k = 0; k < nab; ++k) m2 = fmax(m2, fabs(buf[k * nab + k]));
            double g = sqrt(m2);
            Gp[((size_t)sa * ns + sb) * 64 + i * Kb + j] = g;
            Gp[((size_t)sb * ns + sa) * 64 + j * Ka + i] = g;
          }
      }
    free(buf);
    or_work_free(&w);
  }
}

int oracle_schwarz(int nshell, const double *center, const int32_t *l, const int32_t *nprim,
                   const int32_t *prim_off, const double *exps, const double *coefs, double *G,
                   double *Gp) {
  or_basis B = {nshell, center, l, nprim, prim_off, exps, coefs};
  or_ctx X;
  if (or_ctx_init(&X, &B)) return 1;
  or_schwarz(&X, G, Gp);
  or_ctx_free(&X);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* J and K                                                                    */
/* ------------------------------------------------------------------------- */
/* Neumaier accumulator pair (sum, compensation) */
static inline void nsum(double *s, double *c, double x) {
  double t = *s + x;
  if (fabs(*s) >= fabs(x))
    *c += (*s - t) + x;
  else
    *c += (x - t) + *s;
  *s = t;
}

/* Screening modes: none; Schwarz; Schwarz x density max over the six Fock
 * blocks of the fused J/K build; over the two blocks that feed J (D_ab, D_cd)
 * or over the four that feed K (D_ac, D_ad, D_bc, D_bd) -- the separate J and
 * K builds of Sec. 4.2 and 4.3 each weight a quartet by the density elements
 * it is contracted with. */
enum { OR_SCREEN_NONE = 0, OR_SCREEN_SCHWARZ = 1, OR_SCREEN_DENSITY = 2, OR_SCREEN_DENSITY_J = 3,
       OR_SCREEN_DENSITY_K = 4 };

typedef struct {
  or_ctx X;
  double *G, *Gp, *Dsh;
  double tau;
  int mode;
} or_jk_setup;

static int or_setup(or_jk_setup *S, const or_basis *B, const double *Dm, double tau, int mode,
                    double eps_p) {
  if (or_ctx_init(&S->X, B)) return 1;
  int ns = B->nshell, N = S->X.nbf;
  S->G = (double *)calloc((size_t)ns * ns, sizeof(double));
  S->Gp = (double *)calloc((size_t)ns * ns * 64, sizeof(double));
  S->Dsh = (double *)calloc((size_t)ns * ns, sizeof(double));
  S->tau = tau;
  S->mode = mode;
  if (mode != OR_SCREEN_NONE || eps_p > 0.0) or_schwarz(&S->X, S->G, S->Gp);
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b) {
      double mx = 0.0;
      for (int i = S->X.bf_off[a]; i < S->X.bf_off[a + 1]; ++i)
        for (int j = S->X.bf_off[b]; j < S->X.bf_off[b + 1]; ++j) mx = fmax(mx, fabs(Dm[(size_t)i * N + j]));
      S->Dsh[(size_t)a * ns + b] = mx;
    }
  if (eps_p > 0.0) {
    double gmax = 0.0;
    for (size_t k = 0; k < (size_t)ns * ns; ++k) gmax = fmax(gmax, S->G[k]);
    S->X.keep = (uint64_t *)malloc(sizeof(uint64_t) * ns * ns);
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns; ++b) {
        uint64_t m = 0;
        int Ka = B->nprim[a], Kb = B->nprim[b];
        for (int i = 0; i < Ka; ++i)
          for (int j = 0; j < Kb; ++j)
            if (!(S->Gp[((size_t)a * ns + b) * 64 + i * Kb + j] * gmax < tau * eps_p)) m |= (uint64_t)1 << (i * Kb + j);
        S->X.keep[(size_t)a * ns + b] = m;
      }
  }
  return 0;
}

static void or_setup_free(or_jk_setup *S) {
  free(S->G);
  free(S->Gp);
  free(S->Dsh);
  or_ctx_free(&S->X);
}

/* max |D| over the shell blocks of (ab|cd) the screening mode weights with:
 * all six (Sec. 3.2), the J pair {ab, cd} or the K four {ac, ad, bc, bd} */
static double or_dmax(const or_jk_setup *S, int a, int b, int c, int d) {
  int ns = S->X.B->nshell;
  const double *Q = S->Dsh;
  double dj = fmax(Q[(size_t)a * ns + b], Q[(size_t)c * ns + d]);
  double dk = fmax(fmax(Q[(size_t)a * ns + c], Q[(size_t)a * ns + d]),
                   fmax(Q[(size_t)b * ns + c], Q[(size_t)b * ns + d]));
  if (S->mode == OR_SCREEN_DENSITY_J) return dj;
  if (S->mode == OR_SCREEN_DENSITY_K) return dk;
  return fmax(dj, dk);
}

/* The contracted quartet (ab|cd) of a J/K loop: density-weighted primitive
 * quartet screening with the pruning factor eps_p (mode M2 only). */
static void or_jk_quartet(const or_jk_setup *S, or_work *w, int a, int b, int c, int d, double eps_p,
                          double *eri) {
  int ns = S->X.B->nshell;
  if (S->mode >= OR_SCREEN_DENSITY && eps_p > 0.0)
    or_shell_quartet(&S->X, w, a, b, c, d, -1, -1, S->Gp + ((size_t)a * ns + b) * 64,
                     S->Gp + ((size_t)c * ns + d) * 64, or_dmax(S, a, b, c, d), S->tau * eps_p, eri);
  else
    or_shell_quartet(&S->X, w, a, b, c, d, -1, -1, NULL, NULL, 0.0, 0.0, eri);
}

/* 1 if the quartet (ab|cd) is screened out */
static int or_screened(const or_jk_setup *S, int a, int b, int c, int d) {
  int ns = S->X.B->nshell;
  if (S->mode == OR_SCREEN_NONE) return 0;
  double g = S->G[(size_t)a * ns + b] * S->G[(size_t)c * ns + d];
  if (S->mode == OR_SCREEN_SCHWARZ) return g < S->tau;
  double dm = or_dmax(S, a, b, c, d);
  /* Sec. 3.2 applies both tests: batches whose Schwarz product is below tau
   * are never launched, and inside the kernel G_ab G_cd Dmax < tau skips. */
  return g < S->tau || g * dm < S->tau;
}

/*
 * Full J and K.  mode: 0 none, 1 Schwarz (G_ab G_cd < tau), 2 Schwarz x
 * six-block density max, 3 / 4 Schwarz x the J / K blocks' density max (only
 * J / only K is then meaningful).  eps_p > 0 enables primitive-pair pruning
 * and (modes 2-4) primitive-quartet screening with that mode's density max.
 * symmetric != 0 loops over unique quartets with explicit 8-fold scatter,
 * otherwise over all ordered quartets (N^4 reference used to validate the
 * scatter on small cases).  Returns 0 on success.
 */
static int or_jk_impl(int nshell, const double *center, const int32_t *l, const int32_t *nprim,
                      const int32_t *prim_off, const double *exps, const double *coefs,
                      const double *Dm, double tau, int mode, double eps_p, int symmetric,
                      int nthreads, int stride, double *J, double *K, double *neri) {
  or_basis B = {nshell, center, l, nprim, prim_off, exps, coefs};
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  or_jk_setup S;
  if (or_setup(&S, &B, Dm, tau, mode, eps_p)) return 1;
  int N = S.X.nbf, ns = nshell;
  const int *off = S.X.bf_off;
  size_t NN = (size_t)N * N;
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  double *acc = (double *)calloc(NN * 4 * nthr, sizeof(double)); /* J,cJ,K,cK per thread */
  /* list of shell pairs */
  int npair = symmetric ? ns * (ns + 1) / 2 : ns * ns;
  int *pa = (int *)malloc(sizeof(int) * npair), *pb = (int *)malloc(sizeof(int) * npair);
  {
    int k = 0;
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < (symmetric ? a + 1 : ns); ++b) {
        pa[k] = a;
        pb[k] = b;
        ++k;
      }
  }
  double cnt = 0.0;
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double *Jt = acc + NN * 4 * tid, *Jc = Jt + NN, *Kt = Jc + NN, *Kc = Kt + NN;
    or_work w;
    or_work_alloc(&w);
    double *eri = (double *)malloc(sizeof(double) * 10000);
#pragma omp for schedule(dynamic, 1) reduction(+ : cnt)
    for (int p1 = 0; p1 < npair; ++p1) {
      if (p1 % stride) continue;
      int a = pa[p1], b = pb[p1];
      for (int p2 = 0; p2 < (symmetric ? p1 + 1 : npair); ++p2) {
        int c = pa[p2], d = pb[p2];
        int na = off[a + 1] - off[a], nb = off[b + 1] - off[b], nc = off[c + 1] - off[c],
            nd = off[d + 1] - off[d];
        if (S.G[(size_t)a * ns + b] * S.G[(size_t)c * ns + d] >= tau) cnt += (double)na * nb * nc * nd;
        if (or_screened(&S, a, b, c, d)) continue;
        or_jk_quartet(&S, &w, a, b, c, d, eps_p, eri);
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb; ++j)
            for (int k = 0; k < nc; ++k)
              for (int m = 0; m < nd; ++m) {
                double v = eri[((i * nb + j) * nc + k) * nd + m];
                int mu = off[a] + i, nu = off[b] + j, la_ = off[c] + k, si = off[d] + m;
                if (!symmetric) {
                  nsum(&Jt[(size_t)mu * N + nu], &Jc[(size_t)mu * N + nu], v * Dm[(size_t)la_ * N + si]);
                  nsum(&Kt[(size_t)mu * N + la_], &Kc[(size_t)mu * N + la_], v * Dm[(size_t)nu * N + si]);
                  continue;
                }
                /* function-level canonical representative of the 8 permutations */
                if (a == b && nu > mu) continue;
                if (c == d && si > la_) continue;
                if (a == c && b == d) {
                  long long i1 = (long long)mu * N + nu, i2 = (long long)la_ * N + si;
                  if (i2 > i1) continue;
                }
                int t[8][4] = {{mu, nu, la_, si}, {nu, mu, la_, si}, {mu, nu, si, la_}, {nu, mu, si, la_},
                               {la_, si, mu, nu}, {si, la_, mu, nu}, {la_, si, nu, mu}, {si, la_, nu, mu}};
                for (int q = 0; q < 8; ++q) {
                  int dup = 0;
                  for (int r = 0; r < q; ++r)
                    if (t[r][0] == t[q][0] && t[r][1] == t[q][1] && t[r][2] == t[q][2] && t[r][3] == t[q][3]) {
                      dup = 1;
                      break;
                    }
                  if (dup) continue;
                  int P = t[q][0], Q = t[q][1], R = t[q][2], T = t[q][3];
                  nsum(&Jt[(size_t)P * N + Q], &Jc[(size_t)P * N + Q], v * Dm[(size_t)R * N + T]);
                  nsum(&Kt[(size_t)P * N + R], &Kc[(size_t)P * N + R], v * Dm[(size_t)Q * N + T]);
                }
              }
      }
    }
    free(eri);
    or_work_free(&w);
  }
  for (size_t k = 0; k < NN; ++k) {
    double js = 0.0, jc = 0.0, ks = 0.0, kc = 0.0;
    for (int t = 0; t < nthr; ++t) {
      const double *base = acc + NN * 4 * t;
      nsum(&js, &jc, base[k]);
      nsum(&js, &jc, base[NN + k]);
      nsum(&ks, &kc, base[2 * NN + k]);
      nsum(&ks, &kc, base[3 * NN + k]);
    }
    J[k] = js + jc;
    K[k] = ks + kc;
  }
  free(acc);
  free(pa);
  free(pb);
  or_setup_free(&S);
  if (neri) *neri = cnt;
  return 0;
}

int oracle_jk(int nshell, const double *center, const int32_t *l, const int32_t *nprim,
              const int32_t *prim_off, const double *exps, const double *coefs, const double *Dm,
              double tau, int mode, double eps_p, int symmetric, int nthreads, double *J,
              double *K) {
  return or_jk_impl(nshell, center, l, nprim, prim_off, exps, coefs, Dm, tau, mode, eps_p, symmetric,
                    nthreads, 1, J, K, NULL);
}

/* The symmetric J/K loop restricted to outer pairs p1 with p1 % stride == 0
 * (a bounded sample of the full build, for CPU timing); *neri receives the
 * number of Cartesian ERIs in the sampled quartets that pass the Schwarz
 * test, the same unit the GPU throughput is quoted in. */
int oracle_jk_sample(int nshell, const double *center, const int32_t *l, const int32_t *nprim,
                     const int32_t *prim_off, const double *exps, const double *coefs,
                     const double *Dm, double tau, int mode, double eps_p, int nthreads, int stride,
                     double *J, double *K, double *neri) {
  if (stride < 1) return 1;
  return or_jk_impl(nshell, center, l, nprim, prim_off, exps, coefs, Dm, tau, mode, eps_p, 1,
                    nthreads, stride, J, K, neri);
}

/*
 * Selected shell-pair blocks of J and K, each computed directly with no
 * permutational symmetry: J_mn (m in a, n in b) over all ordered (c,d), and
 * K_mn over all ordered (c,d) from (a c|b d).  Screening and pruning as in
 * oracle_jk.  Jb/Kb: blocks packed consecutively, each nc(a)*nc(b) row-major.
 */
int oracle_jk_blocks(int nshell, const double *center, const int32_t *l, const int32_t *nprim,
                     const int32_t *prim_off, const double *exps, const double *coefs,
                     const double *Dm, double tau, int mode, double eps_p, int nblk,
                     const int32_t *blk_a, const int32_t *blk_b, int nthreads, double *Jb,
                     double *Kb) {
  or_basis B = {nshell, center, l, nprim, prim_off, exps, coefs};
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  or_jk_setup S;
  if (or_setup(&S, &B, Dm, tau, mode, eps_p)) return 1;
  int N = S.X.nbf, ns = nshell;
  const int *off = S.X.bf_off;
  int *bo = (int *)malloc(sizeof(int) * (nblk + 1));
  bo[0] = 0;
  for (int k = 0; k < nblk; ++k) bo[k + 1] = bo[k] + OR_NC(l[blk_a[k]]) * OR_NC(l[blk_b[k]]);
#pragma omp parallel
  {
    or_work w;
    or_work_alloc(&w);
    double *eri = (double *)malloc(sizeof(double) * 10000);
    double js[100], jc[100], ks[100], kc[100];
#pragma omp for schedule(dynamic, 1)
    for (int k = 0; k < nblk; ++k) {
      int a = blk_a[k], b = blk_b[k];
      int na = OR_NC(l[a]), nb = OR_NC(l[b]);
      memset(js, 0, sizeof(js));
      memset(jc, 0, sizeof(jc));
      memset(ks, 0, sizeof(ks));
      memset(kc, 0, sizeof(kc));
      for (int c = 0; c < ns; ++c)
        for (int d = 0; d < ns; ++d) {
          int nc = OR_NC(l[c]), nd = OR_NC(l[d]);
          if (!or_screened(&S, a, b, c, d)) {
            or_jk_quartet(&S, &w, a, b, c, d, eps_p, eri);
            for (int i = 0; i < na; ++i)
              for (int j = 0; j < nb; ++j)
                for (int p = 0; p < nc; ++p)
                  for (int q = 0; q < nd; ++q)
                    nsum(&js[i * nb + j], &jc[i * nb + j],
                         eri[((i * nb + j) * nc + p) * nd + q] * Dm[(size_t)(off[c] + p) * N + off[d] + q]);
          }
          if (!or_screened(&S, a, c, b, d)) {
            /* (a c | b d): K_ij += (i p | j q) D_pq */
            or_jk_quartet(&S, &w, a, c, b, d, eps_p, eri);
            for (int i = 0; i < na; ++i)
              for (int p = 0; p < nc; ++p)
                for (int j = 0; j < nb; ++j)
                  for (int q = 0; q < nd; ++q)
                    nsum(&ks[i * nb + j], &kc[i * nb + j],
                         eri[((i * nc + p) * nb + j) * nd + q] * Dm[(size_t)(off[c] + p) * N + off[d] + q]);
          }
        }
      for (int t = 0; t < na * nb; ++t) {
        Jb[bo[k] + t] = js[t] + jc[t];
        Kb[bo[k] + t] = ks[t] + kc[t];
      }
    }
    free(eri);
    or_work_free(&w);
  }
  free(bo);
  or_setup_free(&S);
  return 0;
}

/*
 * Counts of symmetry-unique contracted shell quartets and Cartesian ERIs that
 * pass the Schwarz test G_ab G_cd >= tau (the throughput unit), plus the same
 * counts after the six-block density test when Dm != NULL.
 * out[0] = quartets (Schwarz), out[1] = ERIs (Schwarz),
 * out[2] = quartets (density), out[3] = ERIs (density).
 */
int oracle_count(int nshell, const double *center, const int32_t *l, const int32_t *nprim,
                 const int32_t *prim_off, const double *exps, const double *coefs,
                 const double *Dm, double tau, double *out) {
  or_basis B = {nshell, center, l, nprim, prim_off, exps, coefs};
  or_jk_setup S;
  if (or_setup(&S, &B, Dm, tau, OR_SCREEN_DENSITY, 0.0)) return 1;
  int ns = nshell;
  double q1 = 0, e1 = 0, q2 = 0, e2 = 0;
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b <= a; ++b)
      for (int c = 0; c <= a; ++c)
        for (int d = 0; d <= (c == a ? b : c); ++d) {
          double n = (double)OR_NC(l[a]) * OR_NC(l[b]) * OR_NC(l[c]) * OR_NC(l[d]);
          if (S.G[(size_t)a * ns + b] * S.G[(size_t)c * ns + d] >= tau) {
            q1 += 1;
            e1 += n;
            if (!or_screened(&S, a, b, c, d)) {
              q2 += 1;
              e2 += n;
            }
          }
        }
  out[0] = q1;
  out[1] = e1;
  out[2] = q2;
  out[3] = e2;
  or_setup_free(&S);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* one-electron integrals                                                      */
/* ------------------------------------------------------------------------- */
/* 1-D overlap table s[i][j], i <= imax, j <= jmax, unnormalised primitives */
static void or_overlap1d(int imax, int jmax, double a, double b, double Ax, double Bx, double s[8][8]) {
  double p = a + b, Px = (a * Ax + b * Bx) / p, XAB = Ax - Bx;
  s[0][0] = sqrt(M_PI / p) * exp(-a * b / p * XAB * XAB);
  for (int i = 0; i <= imax; ++i)
    for (int j = 0; j <= jmax; ++j) {
      if (i == 0 && j == 0) continue;
      double v;
      if (i > 0) {
        v = (Px - Ax) * s[i - 1][j];
        if (i > 1) v += (i - 1) * s[i - 2][j] / (2 * p);
        if (j > 0) v += j * s[i - 1][j - 1] / (2 * p);
      } else {
        v = (Px - Bx) * s[i][j - 1];
        if (j > 1) v += (j - 1) * s[i][j - 2] / (2 * p);
      }
      s[i][j] = v;
    }
}

/* Kinetic energy matrix T = 1/2 sum_x <d_x a | d_x b>, normalised functions. */
int oracle_kinetic(int nshell, const double *center, const int32_t *l, const int32_t *nprim,
                   const int32_t *prim_off, const double *exps, const double *coefs, double *T) {
  or_basis B = {nshell, center, l, nprim, prim_off, exps, coefs};
  or_ctx X;
  if (or_ctx_init(&X, &B)) return 1;
  int N = X.nbf;
  for (int sa = 0; sa < nshell; ++sa)
    for (int sb = 0; sb < nshell; ++sb) {
      int la = l[sa], lb = l[sb], na = OR_NC(la), nb = OR_NC(lb);
      const double *A = center + 3 * sa, *Bc = center + 3 * sb;
      int ba = OR_NH(la - 1) * (la > 0), bb = OR_NH(lb - 1) * (lb > 0);
      for (int ia = 0; ia < na; ++ia)
        for (int ib = 0; ib < nb; ++ib) {
          const int *u = g_cvec[ba + ia], *v = g_cvec[bb + ib];
          double acc = 0.0;
          for (int i = 0; i < nprim[sa]; ++i)
            for (int j = 0; j < nprim[sb]; ++j) {
              double a = exps[prim_off[sa] + i], b = exps[prim_off[sb] + j];
              double s[3][8][8];
              for (int x = 0; x < 3; ++x) or_overlap1d(la + 1, lb + 1, a, b, A[x], Bc[x], s[x]);
              double t = 0.0;
              for (int x = 0; x < 3; ++x) {
                /* d/dx of x^k exp(-a x^2) = k x^(k-1) - 2a x^(k+1) */
                int ka = u[x], kb = v[x];
                double d = 4.0 * a * b * s[x][ka + 1][kb + 1];
                if (ka > 0) d -= 2.0 * b * ka * s[x][ka - 1][kb + 1];
                if (kb > 0) d -= 2.0 * a * kb * s[x][ka + 1][kb - 1];
                if (ka > 0 && kb > 0) d += (double)ka * kb * s[x][ka - 1][kb - 1];
                double o = 1.0;
                for (int y = 0; y < 3; ++y)
                  if (y != x) o *= s[y][u[y]][v[y]];
                t += 0.5 * d * o;
              }
              acc += X.coef[prim_off[sa] + i] * X.coef[prim_off[sb] + j] * t;
            }
          T[(size_t)(X.bf_off[sa] + ia) * N + X.bf_off[sb] + ib] =
              acc * or_cart_norm(u[0], u[1], u[2]) * or_cart_norm(v[0], v[1], v[2]);
        }
    }
  or_ctx_free(&X);
  return 0;
}

/* Nuclear attraction V = -sum_C Z_C <a| 1/|r - C| |b>, normalised functions:
 * Obara-Saika vertical recurrence on the bra with auxiliary orders
 * Theta^(m)(0,0) = (2 pi / p) K_AB F_m(p |PC|^2), then the horizontal
 * recurrence (a|b+1_i) = (a+1_i|b) + AB_i (a|b). */
int oracle_nuclear(int nshell, const double *center, const int32_t *l, const int32_t *nprim,
                   const int32_t *prim_off, const double *exps, const double *coefs, int natom,
                   const double *Z, const double *xyz, double *V) {
  or_basis B = {nshell, center, l, nprim, prim_off, exps, coefs};
  or_ctx X;
  if (or_ctx_init(&X, &B)) return 1;
  int N = X.nbf;
  double th[OR_NHE][OR_MMAX + 1];
  double cont[OR_NHE];
  double hr[OR_NHE][OR_NH(OR_LMAX)];
  for (int sa = 0; sa < nshell; ++sa)
    for (int sb = 0; sb < nshell; ++sb) {
      int la = l[sa], lb = l[sb], L = la + lb;
      const double *A = center + 3 * sa, *Bc = center + 3 * sb;
      double AB[3], AB2 = 0.0;
      for (int x = 0; x < 3; ++x) {
        AB[x] = A[x] - Bc[x];
        AB2 += AB[x] * AB[x];
      }
      for (int e = 0; e < OR_NH(L); ++e) cont[e] = 0.0;
      for (int i = 0; i < nprim[sa]; ++i)
        for (int j = 0; j < nprim[sb]; ++j) {
          double a = exps[prim_off[sa] + i], b = exps[prim_off[sb] + j], p = a + b;
          double P[3], PA[3];
          for (int x = 0; x < 3; ++x) {
            P[x] = (a * A[x] + b * Bc[x]) / p;
            PA[x] = P[x] - A[x];
          }
          double cc = X.coef[prim_off[sa] + i] * X.coef[prim_off[sb] + j] * 2.0 * M_PI / p * exp(-a * b / p * AB2);
          for (int c = 0; c < natom; ++c) {
            double PC[3], PC2 = 0.0;
            for (int x = 0; x < 3; ++x) {
              PC[x] = P[x] - xyz[3 * c + x];
              PC2 += PC[x] * PC[x];
            }
            double F[OR_MMAX + 1];
            oracle_boys(L, p * PC2, F);
            for (int m = 0; m <= L; ++m) th[0][m] = cc * F[m];
            for (int ie = 1; ie < OR_NH(L); ++ie) {
              int v[3] = {g_cvec[ie][0], g_cvec[ie][1], g_cvec[ie][2]};
              int k = v[0] > 0 ? 0 : (v[1] > 0 ? 1 : 2);
              v[k] -= 1;
              int e1 = g_cidx[v[0]][v[1]][v[2]], nk = v[k], e2 = -1;
              if (nk > 0) {
                v[k] -= 1;
                e2 = g_cidx[v[0]][v[1]][v[2]];
              }
              int deg = g_cvec[ie][0] + g_cvec[ie][1] + g_cvec[ie][2];
              for (int m = 0; m <= L - deg; ++m) {
                double val = PA[k] * th[e1][m] - PC[k] * th[e1][m + 1];
                if (e2 >= 0) val += nk / (2.0 * p) * (th[e2][m] - th[e2][m + 1]);
                th[ie][m] = val;
              }
            }
            for (int e = 0; e < OR_NH(L); ++e) cont[e] -= Z[c] * th[e][0];
          }
        }
      /* HRR: hr[e][b] = (e|b) for |e| in [la, la+lb-|b|] */
      for (int e = OR_NH(la - 1) * (la > 0); e < OR_NH(L); ++e) hr[e][0] = cont[e];
      for (int jb = 1; jb < OR_NH(lb); ++jb) {
        int v[3] = {g_cvec[jb][0], g_cvec[jb][1], g_cvec[jb][2]};
        int bdeg = v[0] + v[1] + v[2];
        int k = v[0] > 0 ? 0 : (v[1] > 0 ? 1 : 2);
        v[k] -= 1;
        int bm = g_cidx[v[0]][v[1]][v[2]];
        for (int e = OR_NH(la - 1) * (la > 0); e < OR_NH(L - bdeg); ++e) {
          int av[3] = {g_cvec[e][0], g_cvec[e][1], g_cvec[e][2]};
          av[k] += 1;
          int ep = g_cidx[av[0]][av[1]][av[2]];
          hr[e][jb] = hr[ep][bm] + AB[k] * hr[e][bm];
        }
      }
      int ba = OR_NH(la - 1) * (la > 0), bb = OR_NH(lb - 1) * (lb > 0);
      for (int ia = 0; ia < OR_NC(la); ++ia)
        for (int ib = 0; ib < OR_NC(lb); ++ib) {
          const int *u = g_cvec[ba + ia], *w = g_cvec[bb + ib];
          V[(size_t)(X.bf_off[sa] + ia) * N + X.bf_off[sb] + ib] =
              hr[ba + ia][bb + ib] * or_cart_norm(u[0], u[1], u[2]) * or_cart_norm(w[0], w[1], w[2]);
        }
    }
  or_ctx_free(&X);
  return 0;
}
