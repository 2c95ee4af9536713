// Internal definitions of the GB300 J/K builder: constants, index helpers,
// device-side data layout and the shell-pair handle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/fock.h"

namespace fk {

constexpr int LMAX = 3;             // f functions
constexpr int LTOT = 4 * LMAX;      // largest total angular momentum of a quartet
constexpr int NCLASS = 10;          // pair classes (la >= lb)
constexpr int MAXPRIM = 8;          // primitives per shell
constexpr int MAXCP = 100;          // Cartesian pairs of an (f,f) pair
constexpr int NHMAX = 455;          // Hermite functions with t+u+v <= 12

// Boys table: F_k(T_i), T_i = i*h, k = 0..BOYS_NORD-1, Taylor expansion of
// order BOYS_TAYLOR about the nearest grid point; T >= BOYS_TMAX uses the
// asymptotic form F_0 = sqrt(pi/T)/2 with upward recursion.
constexpr int BOYS_TAYLOR = 8;                 // terms k = 0..7
constexpr int BOYS_NORD = LTOT + BOYS_TAYLOR;  // orders 0..19
constexpr double BOYS_H = 1.0 / 16.0;
constexpr double BOYS_INVH = 16.0;
constexpr double BOYS_TMAX = 64.0;
constexpr int BOYS_NGRID = 1025;               // T_i for i = 0..1024

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
__host__ __device__ constexpr int nherm(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
__host__ __device__ constexpr int pair_class(int la, int lb) { return la * (la + 1) / 2 + lb; }

// Compact index of the Hermite (or Cartesian) exponent vector (t,u,v):
// ordered by degree t+u+v, then t descending, then u descending.
__host__ __device__ inline int hidx(int t, int u, int v) {
  int d = t + u + v, r = d - t;
  return d * (d + 1) * (d + 2) / 6 + r * (r + 1) / 2 + (r - u);
}

// Cartesian component i (0..ncart(l)-1) of a shell of angular momentum l.
__host__ __device__ inline void cart_comp(int l, int i, int &x, int &y, int &z) {
  int k = 0;
  while (i > k) {
    i -= k + 1;
    ++k;
  }
  x = l - k;
  y = k - i;
  z = i;
}

// Primitive-pair centre and exponent (Px, Py, Pz, zeta), one 32-byte load.
struct __align__(32) PZ {
  double x, y, z, w;
};

// Per-class constant tables, copied into shared memory by the kernels
// (16-byte aligned so its size is a whole number of 16-byte words).
struct alignas(16) ClassTables {
  int16_t eoff[NCLASS][MAXCP + 1];   // E offset of Cartesian pair k within a primitive pair block
  int16_t nE[NCLASS];                // E doubles per primitive pair
  uint8_t comp[LMAX + 1][10][3];     // Cartesian components per shell
  uint8_t hvec[NHMAX][3];            // (t,u,v) of compact Hermite index
};

// Device view of a handle's pair data (plain pointers, passed by value).
struct DevPairs {
  // shells
  const double *sxyz;  // [3*nshell]
  const int *sbf;      // first basis function
  const int *sl;       // angular momentum
  // contracted pairs, sorted (class, contraction bucket, G descending)
  const int2 *ab;      // canonical shells (la >= lb; a >= b when la == lb)
  const double *G;     // Schwarz factor G_ab
  const int2 *prim;    // (first primitive pair, count)
  const int *cls;      // pair class
  // primitive pairs
  const PZ *pz;        // (Px, Py, Pz, zeta)
  const float4 *pf;    // the same in FP32 (grid indices, seeds)
  const double *U;     // U_P sqrt(zeta) (2/sqrt(pi))^(1/2), already folded into E (kept for reference)
  const int *eoff;     // offset of the primitive pair's E block
  const double *E;     // Hermite coefficients (Cartesian normalisation and U folded in)
  const double *Gp;    // primitive Schwarz factor G_[ab]; each pair's primitives sorted by it, descending
  const float *Gpf;    // the same rounded to FP32
  // FP32 copies for the mixed-precision path and the FP32 screening pre-test
  const float *Gf;     // G_ab rounded to FP32
  const float *shl;    // shell centres as FP32 hi/lo pairs: [6*s] = hx hy hz lx ly lz
  const float4 *paf;   // (P - A, zeta) with A the first shell of the canonical pair
  const float *Uf;     // U as above, FP32
  const float *Ef;     // Hermite coefficients, FP32
  const int *smol;     // shell -> molecule of a batch (null for one molecule)
  const int *satom;    // shell -> atom (shells on one atom share an index)
  const float *Gn;     // nshell^2: n_z G_xz for kept pairs (x, z), else 0 (GDG bound)
  const float2 *sRG;   // per shell: radius R_s and largest Schwarz factor G_s of its kept pairs
  int nshell, nbf, npair;
  int nprim_total;
  long long nE_total;
};

// Per-molecule entry of a batched build (device table, rewritten per call).
struct MolEntry {
  const double *D;
  double *J;
  double *K;
  const float *Df;     // FP32 copy of D (mixed path) or null
  long long dsh_off;   // offset of the molecule's nshell^2 block maxima
  long long n2_off;    // offset of the molecule's N^2 block in packed per-call arrays
  int N, s0, ns, pad;  // functions, first shell, shells
};

// Host arrays mirroring DevPairs (the compact, sorted data of a handle).
struct Staging {
  std::vector<double> sxyz;
  std::vector<int> sbf, sl;
  std::vector<int2> ab;
  std::vector<double> G;
  std::vector<int2> prim;
  std::vector<int> cls;
  std::vector<PZ> pz;
  std::vector<float4> pf;
  std::vector<double> U;
  std::vector<int> eoff;
  std::vector<double> E;
  std::vector<double> Gp;
  std::vector<float> Gpf;
  std::vector<float4> paf;
  std::vector<float> Uf, Ef, Gf, shl;
  std::vector<int> smol;
  std::vector<int> satom;
  std::vector<float2> sRG;
  std::vector<float> Gn;
};

// One unit of work: bra pair index, ket pair index range [k0, k1).
struct Unit {
  int bra, k0, k1, pad;
};

// Tier tags at or above this mark the per-class-pair group tiers of the
// FP32 register kernels (tag - kReg32Tag = bra class * NCLASS + ket class).
constexpr int kReg32Tag = 1000;

struct Tier {
  int reg_cb = -1;      // >= 0: per-class register kernel for (bra class, ket class)
  int reg_ck = -1;
  int sb = 0;           // scratch bucket of a full-warp group tier
  int tag = 0;          // class pair + 1 when class pairs are launched apart (tuning)
  int mixed = 0;        // 1: mixed-precision build (kernel variant with FP32 paths)
  int r32_cb = -1;      // >= 0: a group tier of one class pair whose FP32 part
  int r32_ck = -1;      //   runs on the FP32 register kernel k_reg32<cb, ck>
  int G;                // lanes per quartet (group kernel)
  int stride;           // scratch doubles per group
  int warps_per_block;
  int blocks;           // persistent grid
  size_t smem;          // dynamic shared memory per block
  int blocks32 = 0;     // the same for the FP32 part of a mixed group tier,
  size_t smem32 = 0;    // whose scratch needs half the bytes (floats)
  int nunits;
  Unit *d_units;
};

}  // namespace fk

struct fock_shellpairs {
  int device = 0;
  int nshell = 0, nbf = 0;
  double tau_build = 0.0, prune_eps = 1e-3;
  fock_opts opts{};
  // host copies (for statistics and tests)
  std::vector<double> h_sxyz;
  std::vector<int> h_sbf, h_sl;
  std::vector<int2> h_ab;
  std::vector<double> h_G;
  std::vector<int2> h_prim;
  std::vector<int> h_cls;
  std::vector<fk::Unit> h_units;      // all tiers, concatenated
  std::vector<int> h_unit_tier;
  fk::Staging host;                   // compact pair data (merged into batch plans)
  std::vector<double> h_R, h_Gs;      // per-shell radius and Schwarz maximum (decay bound)
  int decay_nbins = 0;                // 0.5-bohr distance bins of the decay fit
  unsigned long long serial = 0;      // unique id (batch plan cache key)
  // device allocations
  void *d_block = nullptr;            // one allocation holding all pair arrays
  fk::DevPairs dev{};
  std::vector<fk::Tier> tiers;
  size_t bytes = 0;
};

namespace fk {
// Byte offsets of the per-call scratch of a J/K build in one buffer (256-byte
// aligned parts): shell-block maxima (FP64) at 0, work counters, the FP32
// copy of D (mixed precision), FP32 block maxima, and in the decay-bound
// exchange mode the bounds W, the distance bins and H, Lambda.  (api.cu)
struct ScratchLayout {
  size_t cnt_off = 0, df_off = 0, dshf_off = 0, w_off = 0, bins_off = 0, hl_off = 0, t_off = 0, gdg_off = 0,
         total = 0;
};
ScratchLayout scratch_layout(const fock_shellpairs *sp);

// Status of a CUDA runtime result; a failure also sets the text returned by
// fock_last_error ("where: error name (description)").  (api.cu)
fock_status cuda_status(cudaError_t e, const char *where);
// FOCK_SYNC_CHECK=1 in the environment: synchronise after every launch.
bool sync_each_launch();

// host helpers (host_pairs.cpp)
const ClassTables &class_tables();
const std::vector<double> &boys_table();
void boys_eval_host(int mmax, double T, double *F);
void hermite_1d(int la, int lb, double p, double xpa, double xpb, double *E /*[4][4][7]*/);
int hermite_count(int la, int lb);
void hermite_pair(int la, int lb, double alpha, const double *A, double beta, const double *B,
                  bool cart_norm, double *out);

// Per-call choices of a J/K build besides precision: which matrices are built
// (1 = J, 2 = K, 3 = both) and the decay-bound exchange test (Wsh null: the
// exact test).
struct CallParts {
  int parts = 3;
  const float *Wsh = nullptr;  // nshell^2 decay bounds of the density blocks
  double k_thresh = 0.0;       // tau*
};

// device entry points (kernels.cu)
cudaError_t upload_tables(cudaStream_t st);
const double *dev_boys();
const float *dev_boys_f();
const ClassTables *dev_class_tables();
cudaError_t launch_schwarz(const DevPairs &dp, double *Gpair, double *Gprim, cudaStream_t st);
cudaError_t launch_dprep(const double *D, int nbf, const int *sbf, const int *sl, int nshell,
                         double *Dsh, cudaStream_t st, float *Df = nullptr, float *Dshf = nullptr);
// prim_eps: primitive-quartet screening factor (the handle's prune_eps; 0 = off)
// counter2: work counter of the FP32 part of a group tier in mixed mode (may
// be null when Df is null)
cudaError_t launch_jk_tier(const Tier &t, const DevPairs &dp, const double *D, const double *Dsh,
                           double tau, double prim_eps, double *J, double *K, int *counter, int *counter2,
                           cudaStream_t st, const float *Df = nullptr, double fp32_cutoff = 0.0,
                           const float *Dshf = nullptr, const CallParts &cp = CallParts());
// Decay bound of Sec. 4.3.1 for one density: bins (nbins doubles, zeroed
// here) of the block maxima Dsh of shells on different atoms by centre
// distance (0.5 bohr), the fit into HL[0] = H, HL[1] = Lambda, and the
// per-shell-pair bounds W (nshell^2 floats; null = fit only).  With Gn
// (nshell^2 floats, n_z G_xz over kept pairs), the FP32 block maxima Dshf and
// two nshell^2 float buffers T, GDG, blocks whose GDG bound is below
// k_thresh get W = 0.
cudaError_t launch_decay_bound(const DevPairs &dp, const double *Dsh, int nbins, double *bins, double *HL, float *W,
                               cudaStream_t st, const float *Gn = nullptr, const float *Dshf = nullptr,
                               float *T = nullptr, float *GDG = nullptr, double k_thresh = 0.0);
cudaError_t launch_symmetrize(double *J, double *K, int n, cudaStream_t st);
// batched variants (one launch over every molecule of a batch)
cudaError_t launch_zero_batch(const MolEntry *mt, const long long *n2_prefix, int nmol, long long total,
                              cudaStream_t st);
cudaError_t launch_dprep_batch(const MolEntry *mt, const long long *dsh_prefix, int nmol, long long total,
                               const int *sbf, const int *sl, double *Dsh, float *Dshf, cudaStream_t st);
cudaError_t launch_symmetrize_batch(const MolEntry *mt, const long long *n2_prefix, int nmol, long long total,
                                    cudaStream_t st);
cudaError_t launch_jk_tier_batch(const Tier &t, const DevPairs &dp, const MolEntry *mt, const double *Dsh,
                                 const float *Dshf, double tau, double prim_eps, int *counter, int *counter2,
                                 cudaStream_t st, double fp32_cutoff);
cudaError_t configure_tier(Tier &t);
int read_and_clear_status(cudaStream_t st, int *status);
int read_bounds(long long out[2]);
}  // namespace fk
