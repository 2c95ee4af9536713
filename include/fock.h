/*
 * fock.h -- C ABI of the GB300 Coulomb/exchange (J/K) builder.
 *
 * The library builds, for a contracted Cartesian Gaussian basis up to f
 * functions and a symmetric density matrix D,
 *
 *     J_mn = sum_ls (mn|ls) D_ls,     K_mn = sum_ls (ml|ns) D_ls
 *
 * (arXiv:2407.21445, Sec. 2.2, Eq. fock_build), from two-electron repulsion
 * integrals (Sec. 2.1) evaluated with the McMurchie-Davidson Hermite scheme
 * (Sec. 4.1, Eqs. MD def, EabP def1-3) and a tabulated Boys function
 * (Eq. boys-fn-def), screened with the Cauchy-Schwarz bound (Eqs.
 * cauchy-schwarz 1, 2) weighted by the density (Sec. 3.2).
 *
 * Conventions shared by every entry point
 *   - Geometry in bohr, exponents in bohr^-2.
 *   - Cartesian functions of a shell are ordered x^l, x^(l-1)y, x^(l-1)z, ...,
 *     z^l (x exponent descending, then y descending); each Cartesian function
 *     is normalised to unit self-overlap.
 *   - D, J, K are N x N row-major float64 matrices in device memory, owned by
 *     the caller; J and K are overwritten with full symmetric matrices.
 *   - Work is asynchronous on the given CUDA stream; argument errors are
 *     returned synchronously, device-side errors (non-finite density, a work
 *     queue wait that timed out) are recorded in a device status word read by
 *     fock_stream_status().
 *   - No entry point traps, asserts or aborts on the device.
 */
#ifndef FOCK_H
#define FOCK_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define FOCK_API __attribute__((visibility("default")))
#else
#define FOCK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FOCK_OK = 0,
  FOCK_ERR_INVALID_ARG = 1,    /* null pointer, bad size, bad threshold      */
  FOCK_ERR_UNSUPPORTED_L = 2,  /* angular momentum > 3 or contraction > 8    */
  FOCK_ERR_NONFINITE = 3,      /* NaN/Inf found in the density (device)      */
  FOCK_ERR_OOM = 4,            /* device or host allocation failed           */
  FOCK_ERR_CUDA = 5,           /* a CUDA runtime call failed                 */
  FOCK_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up         */
  FOCK_ERR_NOT_CONVERGED = 7   /* iterative driver did not converge          */
} fock_status;

enum { FOCK_FP64 = 0, FOCK_MIXED = 1 };

/* Exchange screening modes (fock_opts.k_mode). */
enum {
  FOCK_K_EXACT = 0,       /* rigorous density-weighted Schwarz test (Sec. 3.2)     */
  FOCK_K_DECAY_BOUND = 1  /* heuristic decay bound of Sec. 4.3.1: K contributions
                             below k_thresh by H exp(-Lambda r) are not evaluated */
};

/* Basis description: host pointers, caller-owned, read only during
 * fock_shellpairs_build.  Shell s has angular momentum l[s] (0..3), nprim[s]
 * (1..8) primitives whose exponents and raw contraction coefficients (for
 * primitive-normalised Gaussians, Sec. 2.1 Eq. prim) are exps/coefs[prim_off[s]
 * .. prim_off[s]+nprim[s]-1]; centre[3*s..3*s+2] in bohr; atom[s] is the
 * index of the atom carrying the shell (may be NULL). */
typedef struct {
  int32_t nshell;
  const double *center;
  const int32_t *l;
  const int32_t *nprim;
  const int32_t *prim_off;
  const double *exps;
  const double *coefs;
  const int32_t *atom;
} fock_basis_desc;

/* Angular-momentum classes of a shell pair, ss .. ff (l <= 3). */
#define FOCK_NCLASS 10

/* Options; pass NULL for the defaults shown. */
typedef struct {
  int32_t precision;    /* FOCK_FP64 (default) or FOCK_MIXED                     */
  double fp32_cutoff;   /* mixed path: quartets with G_ab G_cd Dmax, and
                           primitive quartets with G_[ab] G_[cd] Dmax, below
                           this bound are evaluated in FP32 (default 1e-5)      */
  double prune_eps;     /* primitive screening (Sec. 3.2, 3.3): primitive pair
                           [ab] dropped when G_[ab] Gmax < tau * prune_eps, and
                           inside a quartet that passes, primitive quartet
                           [ab|cd] skipped when G_[ab] G_[cd] Dmax < tau *
                           prune_eps (Dmax the six-block density maximum)
                           (default 1e-3; 0 disables both)                       */
  int32_t group_override; /* 0 = autotuned per class pair; 1..32 = lanes per
                             quartet forced for every class pair (testing)     */
  int32_t warp_scratch;   /* shared-memory doubles one warp may use for the
                             intermediates of its quartets (0 = default 1536);
                             sets lanes per quartet against occupancy          */
  int32_t reg_max_L;      /* class pairs with total angular momentum up to this
                             use the per-class register kernels (0 = default 4;
                             -1 = none)                                          */
  int32_t tune_isolate;   /* 1: every class pair gets launches of its own, so
                             that its time can be measured (fock_autotune);
                             0 (default): class pairs with the same kernel
                             share one launch                                  */
  int8_t schedule[FOCK_NCLASS * FOCK_NCLASS];
                          /* per class pair {x, y}, entry [min(x,y) * FOCK_NCLASS
                             + max(x,y)] (class index of shell pair (la >= lb):
                             la (la + 1) / 2 + lb, ss = 0 ... ff = 9):
                             0 = the built-in rule; -1 = the per-class register
                             kernel where one exists for the pair (else the
                             built-in rule); 1, 2, 4, 8, 16, 32 = the group
                             kernel with that many lanes per quartet (raised
                             where a warp's scratch would not fit).  Filled by
                             fock_autotune.  Ignored where group_override > 0. */
  int32_t k_mode;         /* FOCK_K_EXACT (default) or FOCK_K_DECAY_BOUND: the
                             exchange part of a quartet is needed when, for one
                             of its four K blocks (x, y), G_ab G_cd
                             H exp(-Lambda max(0, |XY| - R_x - R_y)) >= k_thresh
                             (Sec. 4.3.1: |D| <= H exp(-Lambda r) fitted to the
                             density on every call; R_s the largest distance
                             from shell s to a shell it forms a kept pair with);
                             the Coulomb part keeps the exact test            */
  double k_thresh;        /* tau* of the decay-bound mode (> 0; 5e-6 in the
                             paper's experiments); ignored in FOCK_K_EXACT     */
} fock_opts;

/* sizeof(fock_opts) as compiled into the library (binding layout check). */
FOCK_API int32_t fock_opts_size(void);

typedef struct fock_shellpairs fock_shellpairs; /* opaque, library-owned */

/*
 * Build the shell-pair data for one geometry (Sec. 3.2 batching and
 * primitive screening, Sec. 4.2 sorted pair lists): normalisation,
 * primitive pairs (zeta, P, U_P; Sec. 2.1 Eq. zeta), Hermite expansion
 * coefficients E^{ab}_p (Sec. 4.1 Eqs. EabP def1-3), Schwarz factors G_ab and
 * G_[ab] from diagonal integrals computed on the GPU (Eqs. cauchy-schwarz 1,
 * 2), primitive-pair pruning, and the quartet work lists of pairs binned by
 * angular-momentum class and contraction degree whose Schwarz product is at
 * least schwarz_thresh.
 *   desc, opts: host, read during the call.   schwarz_thresh > 0.
 *   stream: the CUDA stream the build's kernels run on; the call
 *   synchronises that stream before returning.
 *   *out receives a handle owned by the library (free with
 *   fock_shellpairs_free); it is immutable afterwards and may be shared by
 *   calls on several streams.
 * Errors: FOCK_ERR_INVALID_ARG (null pointers, nshell < 1, bad exponents or
 * offsets, threshold <= 0), FOCK_ERR_UNSUPPORTED_L (l > 3, nprim > 8),
 * FOCK_ERR_OOM, FOCK_ERR_CUDA.  On error *out is set to NULL.
 */
FOCK_API fock_status fock_shellpairs_build(const fock_basis_desc *desc, const fock_opts *opts,
                                  double schwarz_thresh, cudaStream_t stream,
                                  fock_shellpairs **out);

/* Release a handle (NULL is accepted).  The caller must ensure no work using
 * it is still in flight. */
FOCK_API fock_status fock_shellpairs_free(fock_shellpairs *sp);

/* Number of Cartesian basis functions N of the handle (-1 for NULL). */
FOCK_API int32_t fock_nbasis(const fock_shellpairs *sp);

/*
 * J and K for one density (Sec. 2.2 Eq. fock_build), one SCF iteration of the
 * direct method (Sec. 2.2): every symmetry-unique contracted shell quartet
 * (Sec. 2.3, 8-fold symmetry) whose density-weighted Schwarz bound
 * G_ab G_cd max(|D_ab|,|D_ac|,|D_ad|,|D_bc|,|D_bd|,|D_cd|) is not below
 * schwarz_thresh (Sec. 3.2) is evaluated and digested into J and K.  Inside
 * such a quartet, a primitive quartet [ab|cd] is skipped when
 * G_[ab] G_[cd] Dmax < schwarz_thresh * prune_eps (Sec. 3.2, 3.3).  With
 * precision FOCK_MIXED, a quartet whose bound is below fp32_cutoff is
 * evaluated in FP32, and inside a quartet at or above it every primitive
 * quartet whose own bound G_[ab] G_[cd] Dmax is below fp32_cutoff is
 * evaluated in FP32; all contributions are accumulated in FP64.
 *   D: device, N x N row-major float64, symmetric (read).
 *   J, K: device, N x N row-major float64 (overwritten).  One of them may be
 *   NULL: then only the other is built, and the density test of a quartet
 *   uses only the blocks that feed it (J: D_ab, D_cd; K: D_ac, D_ad, D_bc,
 *   D_bd), as the paper's separate J and K schemes do (Sec. 4.2, 4.3).
 *   schwarz_thresh >= the value the handle was built with.
 *   stream: all work is enqueued on it; no host synchronisation.
 * Per-call scratch (shell-block density maxima, work counters) is taken from
 * the stream-ordered allocator (cudaMallocAsync) and released on the stream.
 * With k_mode FOCK_K_DECAY_BOUND the handle's exchange test is the
 * heuristic decay bound (see fock_opts; H and Lambda are fitted on the device
 * from the shell-block maxima of D on every call).
 * Errors (synchronous): FOCK_ERR_INVALID_ARG (null pointers, J and K both
 * NULL, threshold below the build threshold), FOCK_ERR_OOM, FOCK_ERR_CUDA.  A NaN/Inf in D sets
 * FOCK_ERR_NONFINITE in the status word (fock_stream_status).  With the
 * environment variable FOCK_SYNC_CHECK=1 every launch is followed by a
 * stream synchronisation so that a failure names its kernel
 * (fock_last_error); that mode is for diagnosis only.
 */
FOCK_API fock_status fock_build_jk(const fock_shellpairs *sp, const double *D, double schwarz_thresh,
                          double *J, double *K, cudaStream_t stream);

/*
 * The density decay bound of Sec. 4.3.1 (Eq. density_bound, |D_cd| <=
 * H exp(-Lambda |CD|)) as fock_build_jk fits it in FOCK_K_DECAY_BOUND mode:
 * the shell-block maxima max|D| of every pair of shells on different atoms
 * (atom from fock_basis_desc.atom, or one atom per shell when NULL) are
 * binned by the distance of the shell centres in bins of 0.5 bohr; ln of each
 * bin's maximum is fitted by least squares to ln H - Lambda r (r the bin
 * centre), and ln H is then raised until the line lies above every bin's
 * maximum over the whole bin, so that the bound holds for every such element.
 * Also the per-shell radius R_s (largest centre distance from shell s to a
 * shell it forms a kept pair with, Sec. 4.3.1 read with the condition
 * G >= tau) and G_s (largest Schwarz factor of those pairs).
 *   D: device, N x N row-major float64.  out_HL[0] = H, out_HL[1] = Lambda
 *   (bohr^-1); R, G: host arrays of nshell doubles (either may be NULL).
 * Synchronises the stream.  Errors: FOCK_ERR_INVALID_ARG, FOCK_ERR_CUDA.
 */
FOCK_API fock_status fock_decay_bound(const fock_shellpairs *sp, const double *D, double out_HL[2], double *R,
                                      double *G, cudaStream_t stream);

/*
 * fock_build_jk without any device allocation.  The paper has no counterpart:
 * this entry point is for callers that must not allocate device memory while
 * they run -- services that reserve their whole memory budget at start-up,
 * applications whose allocator policy forbids the CUDA runtime's
 * stream-ordered pool, real-time loops where an allocation could stall.
 * Arguments, layouts, errors and results are those of fock_build_jk, in both
 * precisions (the same kernels run with the same inputs).  The per-call
 * scratch lives in a fixed 4 MiB array inside the library, which every GPU
 * that loads the library keeps until the process exits.  A call needs
 * 12 nshell^2 bytes (shell-block density maxima in FP64 and FP32), plus
 * 4 N^2 bytes with FOCK_MIXED (the FP32 copy of D), plus 12 nshell^2 bytes
 * and 8 bytes per 0.5 bohr of the molecule's extent with FOCK_K_DECAY_BOUND
 * (the bounds and the GDG products), plus a few hundred bytes of work
 * counters: FP64 handles in the exact exchange mode fit up to 591 shells.
 * Handles that do not fit return FOCK_ERR_INVALID_ARG without doing any work.
 * J or K may be NULL as in fock_build_jk.  Every call looks
 * up the array's device address (cudaGetSymbolAddress); the first call on
 * each device also loads the library's device code there, so make that first
 * call before any stream capture.  Every call uses the same array: calls
 * whose GPU work can overlap (other streams, other host threads) race on it
 * and must be serialised by the caller.  No cudaMalloc, cudaMallocAsync or
 * cudaFree is called.
 */
FOCK_API fock_status fock_build_jk_noalloc(const fock_shellpairs *sp, const double *D, double schwarz_thresh,
                                           double *J, double *K, cudaStream_t stream);

/*
 * J and K for nmol independent molecules in one pass: bases[i], D[i], J[i],
 * K[i] as in fock_build_jk (all device pointers; the pointer arrays themselves
 * are host memory read during the call).  All handles must have been built
 * with the same options and threshold.  The molecules' work lists are merged
 * per kernel tier (one launch per tier covers every molecule); the merged
 * plan is cached per list of handles (the four most recent lists) and its
 * launches are captured once into a CUDA graph on a library-owned stream,
 * which is ordered after `stream` and `stream` after it by events.  The
 * result is the same as nmol calls of fock_build_jk.
 * Errors: FOCK_ERR_INVALID_ARG (null pointers, nmol < 0, handles with
 * different options), FOCK_ERR_OOM, FOCK_ERR_CUDA; nmol == 0 does nothing.
 */
FOCK_API fock_status fock_build_jk_batched(const fock_shellpairs *const *bases, int32_t nmol,
                                  const double *const *D, double schwarz_thresh,
                                  double *const *J, double *const *K, cudaStream_t stream);

/*
 * Work statistics of the handle for the given density and threshold,
 * computed on the host from the handle's pair data and a host copy of the
 * shell-block density maxima:
 *   out[0] symmetry-unique contracted quartets passing Schwarz (G_ab G_cd >= tau)
 *   out[1] Cartesian ERIs in those quartets (throughput unit)
 *   out[2] quartets also passing the density-weighted test (evaluated)
 *   out[3] Cartesian ERIs in evaluated quartets
 *   out[4] primitive quartets evaluated (after primitive-quartet screening)
 *   out[5] modelled FP64 floating-point operations of the evaluated work, an
 *          FMA counting 2 (per-class Hermite-scheme counts: primitive-quartet
 *          setup, Boys, R recursion, ket and bra Hermite transforms,
 *          digestion)
 *   out[6] primitive pairs kept after pruning
 *   out[7] contracted pairs kept
 *   out[8] evaluated quartets taken by the FP32 path (mixed precision)
 *   out[9] modelled floating-point operations run in FP32: those FP32
 *          quartets, plus the primitive quartets below the cutoff inside the
 *          FP64 ones (mixed precision)
 * D: host, N x N row-major float64.  Synchronous.
 */
FOCK_API fock_status fock_work_stats(const fock_shellpairs *sp, const double *D_host,
                            double schwarz_thresh, double out[10]);

/* Number of kernels one fock_build_jk call on this handle launches (density
 * preparation, one persistent ERI/digestion kernel per work tier -- two for a
 * group-kernel tier in mixed precision, its FP64 and its FP32 part -- and the
 * final symmetrisation); -1 for NULL.  Host only. */
FOCK_API int32_t fock_kernels_per_build(const fock_shellpairs *sp);

/*
 * Measured per-class-pair schedule (no counterpart in the paper, whose kernels
 * use fixed block sizes of 64 or 128 threads per class, Sec. 4.2).  For each
 * candidate schedule (the register kernel, group kernels of 1, 2, 4, 8, 16, 32
 * lanes per quartet) the workload is planned with tune_isolate = 1 and built
 * `reps` times with CUDA events around every launch; each class pair present
 * then takes the candidate with the smallest time if it beats the built-in
 * rule by more than 3%.  Finally the whole build is timed with the base and
 * the tuned schedule (tune_isolate = 0, `reps` builds each, median) and the
 * faster of the two is returned.
 *   descs[nmol], D[nmol]: the workload (host basis descriptions as
 *   fock_shellpairs_build; device N_i x N_i row-major float64 densities).
 *   nmol == 1 times fock_build_jk, nmol > 1 times fock_build_jk_batched
 *   (the batched path without its graph while measuring class pairs).
 *   base: starting options (NULL = defaults); its schedule entries other
 *   than 0 are kept where no candidate beats them.  schwarz_thresh as for
 *   fock_shellpairs_build and fock_build_jk.  reps in 1..100.
 *   *tuned: receives base with the chosen schedule (tune_isolate = 0).
 *   ms[0], ms[1] (may be NULL): median build time in milliseconds with the
 *   base and with the tuned schedule; *tuned is the faster of the two.
 *   pair_ms (may be NULL, FOCK_NCLASS * FOCK_NCLASS doubles): the time of
 *   each class pair with the base schedule, launched apart (the smallest
 *   over the reps), at the index of the schedule entry; 0 where absent.
 * Allocates and frees its own J, K and handles; synchronises `stream`;
 * takes seconds (7 candidate plans, (reps + 1) builds each).
 * Errors: as fock_shellpairs_build and fock_build_jk; FOCK_ERR_INVALID_ARG
 * for null pointers, nmol < 1 or reps outside 1..100.
 */
FOCK_API fock_status fock_autotune(const fock_basis_desc *const *descs, int32_t nmol, const double *const *D,
                                   const fock_opts *base, double schwarz_thresh, int32_t reps,
                                   cudaStream_t stream, fock_opts *tuned, double *ms, double *pair_ms);

/*
 * FP64 one-electron integrals for the RHF driver (Sec. 2.2: F = h + J - K/2,
 * h = T + V): overlap S, kinetic T and nuclear attraction V over the same
 * normalised Cartesian basis as the J/K build, by the McMurchie-Davidson
 * Hermite expansion (Sec. 4.1) with the tabulated Boys function.
 *   desc: host basis (as fock_shellpairs_build).  natom nuclei with charges
 *   Z[natom] and positions xyz[3*natom] (bohr), host.
 *   S, T, V: device, N x N row-major float64, overwritten (full, symmetric).
 * Synchronises the stream.  Errors: FOCK_ERR_INVALID_ARG,
 * FOCK_ERR_UNSUPPORTED_L, FOCK_ERR_OOM, FOCK_ERR_CUDA.
 */
FOCK_API fock_status fock_one_electron(const fock_basis_desc *desc, int32_t natom, const double *Z,
                                       const double *xyz, double *S, double *T, double *V, cudaStream_t stream);

/*
 * Atom-pair MLP of the learned SCF guess (no counterpart in the paper; the
 * SCF extension).  Three dense layers nin -> nhidden -> nhidden -> nout with
 * SiLU activations; BF16 weights, FP32 activations, FP32 accumulation; FP32
 * master parameters with Adam.  Parameter vector layout (FP32):
 * W1[nhidden][nin], b1[nhidden], W2[nhidden][nhidden], b2[nhidden],
 * W3[nout][nhidden], b3[nout].  All tensors are row-major device arrays
 * owned by the caller unless stated; the handle owns parameters, gradients,
 * optimiser state and activation buffers for max_batch rows.
 */
typedef struct fock_mlp fock_mlp;
FOCK_API fock_status fock_mlp_create(int32_t nin, int32_t nhidden, int32_t nout, int32_t max_batch, uint64_t seed,
                                     fock_mlp **out);
FOCK_API fock_status fock_mlp_free(fock_mlp *net);
/* number of FP32 parameters (-1 for NULL) */
FOCK_API int64_t fock_mlp_num_params(const fock_mlp *net);
/* copy parameters and/or accumulated gradients to host arrays of num_params floats (either may be NULL) */
FOCK_API fock_status fock_mlp_get_params(const fock_mlp *net, float *host_params, float *host_grads);
FOCK_API fock_status fock_mlp_set_params(fock_mlp *net, const float *host_params);
/* Y[B][nout] = net(X[B][nin]); B <= max_batch; device pointers */
FOCK_API fock_status fock_mlp_forward(fock_mlp *net, const float *X, int32_t B, float *Y, cudaStream_t stream);
/* loss = sum mask (Y - T)^2 / norm over B rows (mask may be NULL); the
 * gradient of the loss is ADDED to the handle's gradient buffer; the loss is
 * written to *loss_host when non-NULL (synchronises the stream). */
FOCK_API fock_status fock_mlp_loss_backward(fock_mlp *net, const float *X, const float *T, const float *mask,
                                            int32_t B, double norm, float *loss_host, cudaStream_t stream);
/* Adam step with decoupled weight decay on the accumulated gradients, then
 * zero the gradients and refresh the BF16 weights. */
FOCK_API fock_status fock_mlp_step(fock_mlp *net, float lr, float beta1, float beta2, float eps, float weight_decay,
                                   cudaStream_t stream);
FOCK_API fock_status fock_mlp_zero_grad(fock_mlp *net, cudaStream_t stream);

/* Synchronise the stream, return and clear the device status word
 * (FOCK_OK if no device-side error was recorded). */
FOCK_API fock_status fock_stream_status(cudaStream_t stream);

/* Description of the most recent CUDA runtime failure seen by the library
 * on the calling thread ("" if none): the failing step and the CUDA error
 * name.  Static thread-local storage, overwritten by the next failure. */
FOCK_API const char *fock_last_error(void);

/* Diagnostic word of a library built with -DFOCK_BOUNDS_CHECK: out[0] is
 * the site of the first failed device-side bounds check (0 = none), out[1]
 * the offending value.  Always {0, 0} in a normal build.  Synchronous. */
FOCK_API fock_status fock_debug_bounds(int64_t out[2]);

/* Human-readable name of a status code (static storage). */
FOCK_API const char *fock_status_string(fock_status st);

/*
 * Host-side inspection of the handle's precomputed tables, for tests (no
 * device work; safe without a GPU once a handle exists):
 * Boys table parameters: out[0] grid step h, out[1] number of grid points,
 * out[2] number of orders stored, out[3] T beyond which the asymptotic form
 * is used.
 */
FOCK_API fock_status fock_boys_table_info(double out[4]);

/*
 * Host evaluation of the library's own tabulated Boys function (same table
 * and Taylor rule the kernels use), F_m(T) for m = 0..mmax into F.
 * For tests of the table against independent evaluations.
 */
FOCK_API fock_status fock_boys_host(int32_t mmax, double T, double *F);

/*
 * Hermite expansion coefficients E^{ab}_{tuv} (Sec. 4.1, Eqs. EabP def1-3)
 * of one primitive pair, as the kernels store them: for every Cartesian pair
 * (a component major, b component minor) the box t<=ax+bx, u<=ay+by,
 * v<=az+bz in t-major order, WITHOUT the Cartesian normalisation factors.
 * out must hold fock_hermite_count(la, lb) doubles.  alpha/A on shell a,
 * beta/B on shell b.  Host only.
 */
FOCK_API int32_t fock_hermite_count(int32_t la, int32_t lb);
FOCK_API fock_status fock_hermite_e(int32_t la, int32_t lb, double alpha, const double *A, double beta,
                           const double *B, double *out);

#ifdef __cplusplus
}
#endif
#endif /* FOCK_H */
