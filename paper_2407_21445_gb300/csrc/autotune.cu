// fock_autotune: per-class-pair schedules chosen by measurement.
//
// A class pair (bra class, ket class) can run on its per-class register
// kernel (where one exists) or on the group-cooperative kernel with 1..32
// lanes per quartet; which is fastest depends on the contraction degrees, the
// screening survival and the occupancy the class reaches, so the choice is
// measured.  Every candidate is planned with tune_isolate = 1 (each class pair
// in launches of its own) and timed with CUDA events around every launch;
// the per-class-pair minima make the schedule, which is then checked against
// the base schedule on whole builds.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fock_impl.h"

namespace fk {
fock_opts default_opts();
bool valid_opts(const fock_opts &o);
fock_status build_jk_events(const fock_shellpairs *sp, const double *D, double schwarz_thresh, double *J,
                            double *K, cudaStream_t stream, const cudaEvent_t *ev);
fock_status batch_tier_times(const fock_shellpairs *const *bases, int nmol, const double *const *D, double tau,
                             double *const *J, double *const *K, int reps, cudaStream_t stream,
                             std::vector<double> &ms_by_tag);
}  // namespace fk

using namespace fk;

namespace {

constexpr int kNPairs = FOCK_NCLASS * FOCK_NCLASS;
constexpr int kCand[] = {-1, 1, 2, 4, 8, 16, 32};

fock_status cuda_st(cudaError_t e) { return e == cudaSuccess ? FOCK_OK : FOCK_ERR_CUDA; }

struct Workload {
  const fock_basis_desc *const *descs;
  int nmol;
  const double *const *D;
  double tau;
  cudaStream_t stream;
  std::vector<double *> J, K;  // device outputs, one pair per molecule
};

struct Handles {
  std::vector<fock_shellpairs *> h;
  ~Handles() {
    for (fock_shellpairs *p : h) fock_shellpairs_free(p);
  }
};

fock_status make_handles(const Workload &w, const fock_opts &o, Handles &out) {
  for (int i = 0; i < w.nmol; ++i) {
    fock_shellpairs *sp = nullptr;
    fock_status s = fock_shellpairs_build(w.descs[i], &o, w.tau, w.stream, &sp);
    if (s != FOCK_OK) return s;
    out.h.push_back(sp);
  }
  return FOCK_OK;
}

// Class-pair times (ms by tag, tag = class pair + 1) of an isolated plan.
fock_status tag_times(Workload &w, const Handles &hs, int reps, std::vector<double> &ms) {
  ms.assign(kNPairs + 1, 0.0);
  if (w.nmol > 1)
    return batch_tier_times(hs.h.data(), w.nmol, w.D, w.tau, w.J.data(), w.K.data(), reps, w.stream, ms);
  const fock_shellpairs *sp = hs.h[0];
  const size_t nt = sp->tiers.size();
  std::vector<cudaEvent_t> ev(nt + 1, nullptr);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i <= nt && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  fock_status s = cuda_st(e);
  std::vector<double> best;
  for (int r = 0; r <= reps && s == FOCK_OK; ++r) {  // run 0 warms up
    s = build_jk_events(sp, w.D[0], w.tau, w.J[0], w.K[0], w.stream, ev.data());
    if (s == FOCK_OK) s = cuda_st(cudaStreamSynchronize(w.stream));
    if (s != FOCK_OK || r == 0) continue;
    std::vector<double> cur(kNPairs + 1, 0.0);
    for (size_t t = 0; t < nt && s == FOCK_OK; ++t) {
      float x = 0.f;
      s = cuda_st(cudaEventElapsedTime(&x, ev[t], ev[t + 1]));
      const int tag = sp->tiers[t].tag;
      if (tag >= 0 && tag <= kNPairs) cur[tag] += x;
    }
    if (best.empty()) best = cur;
    for (int i = 0; i <= kNPairs; ++i) best[i] = std::min(best[i], cur[i]);
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (s == FOCK_OK) ms = best;
  return s;
}

// Median whole-build time (ms) of a plan, `reps` builds after one warm-up.
fock_status build_time(Workload &w, const Handles &hs, int reps, double *ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  fock_status s = cuda_st(e);
  std::vector<float> t;
  for (int r = 0; r <= reps && s == FOCK_OK; ++r) {
    s = cuda_st(cudaEventRecord(e0, w.stream));
    if (s == FOCK_OK) {
      if (w.nmol == 1)
        s = fock_build_jk(hs.h[0], w.D[0], w.tau, w.J[0], w.K[0], w.stream);
      else
        s = fock_build_jk_batched(hs.h.data(), w.nmol, w.D, w.tau, w.J.data(), w.K.data(), w.stream);
    }
    if (s == FOCK_OK) s = cuda_st(cudaEventRecord(e1, w.stream));
    if (s == FOCK_OK) s = cuda_st(cudaEventSynchronize(e1));
    float x = 0.f;
    if (s == FOCK_OK) s = cuda_st(cudaEventElapsedTime(&x, e0, e1));
    if (s == FOCK_OK && r > 0) t.push_back(x);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s != FOCK_OK) return s;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return FOCK_OK;
}

fock_status tune(Workload &w, const fock_opts &base, int reps, fock_opts *tuned, double *ms, double *pair_ms) {
  // the base schedule, class pairs apart
  fock_opts iso = base;
  iso.tune_isolate = 1;
  std::vector<double> t_base;
  {
    Handles hs;
    fock_status s = make_handles(w, iso, hs);
    if (s == FOCK_OK) s = tag_times(w, hs, reps, t_base);
    if (s != FOCK_OK) return s;
  }
  if (pair_ms)
    for (int i = 0; i < kNPairs; ++i) pair_ms[i] = t_base[i + 1];
  std::vector<double> best_t(t_base);
  std::vector<int> best_c(kNPairs, 0);
  for (int c : kCand) {
    fock_opts oc = iso;
    for (int i = 0; i < kNPairs; ++i) oc.schedule[i] = (int8_t)c;
    Handles hs;
    std::vector<double> t;
    fock_status s = make_handles(w, oc, hs);
    if (s == FOCK_OK) s = tag_times(w, hs, reps, t);
    if (s != FOCK_OK) return s;
    for (int i = 0; i < kNPairs; ++i)
      if (t_base[i + 1] > 0.0 && t[i + 1] > 0.0 && t[i + 1] < best_t[i + 1]) {
        best_t[i + 1] = t[i + 1];
        best_c[i] = c;
      }
  }
  fock_opts out = base;
  out.tune_isolate = 0;
  for (int i = 0; i < kNPairs; ++i)
    if (best_c[i] != 0 && best_t[i + 1] < 0.97 * t_base[i + 1]) out.schedule[i] = (int8_t)best_c[i];
  // whole builds: base against tuned
  double ms_base = 0.0, ms_tuned = 0.0;
  {
    fock_opts b = base;
    b.tune_isolate = 0;
    Handles hs;
    fock_status s = make_handles(w, b, hs);
    if (s == FOCK_OK) s = build_time(w, hs, reps, &ms_base);
    if (s != FOCK_OK) return s;
  }
  {
    Handles hs;
    fock_status s = make_handles(w, out, hs);
    if (s == FOCK_OK) s = build_time(w, hs, reps, &ms_tuned);
    if (s != FOCK_OK) return s;
  }
  if (ms) {
    ms[0] = ms_base;
    ms[1] = ms_tuned;
  }
  if (ms_tuned < ms_base) {
    *tuned = out;
  } else {
    *tuned = base;
    tuned->tune_isolate = 0;
  }
  return FOCK_OK;
}

}  // namespace

extern "C" fock_status fock_autotune(const fock_basis_desc *const *descs, int32_t nmol, const double *const *D,
                                     const fock_opts *base, double schwarz_thresh, int32_t reps,
                                     cudaStream_t stream, fock_opts *tuned, double *ms, double *pair_ms) {
  if (!descs || !D || !tuned || nmol < 1 || reps < 1 || reps > 100) return FOCK_ERR_INVALID_ARG;
  for (int i = 0; i < nmol; ++i)
    if (!descs[i] || !D[i]) return FOCK_ERR_INVALID_ARG;
  if (!(schwarz_thresh > 0.0) || !isfinite(schwarz_thresh)) return FOCK_ERR_INVALID_ARG;
  const fock_opts b = base ? *base : default_opts();
  if (!valid_opts(b)) return FOCK_ERR_INVALID_ARG;
  Workload w{descs, nmol, D, schwarz_thresh, stream, {}, {}};
  // J and K of every molecule in one allocation
  std::vector<size_t> off(nmol + 1, 0);
  for (int i = 0; i < nmol; ++i) {
    int n = 0;
    for (int s = 0; s < descs[i]->nshell; ++s) {
      const int l = descs[i]->l[s];
      if (l < 0 || l > LMAX) return FOCK_ERR_UNSUPPORTED_L;
      n += (l + 1) * (l + 2) / 2;
    }
    off[i + 1] = off[i] + 2 * (size_t)n * n;
  }
  double *buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, sizeof(double) * std::max<size_t>(off[nmol], 1));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FOCK_ERR_OOM : FOCK_ERR_CUDA;
  for (int i = 0; i < nmol; ++i) {
    const size_t n2 = (off[i + 1] - off[i]) / 2;
    w.J.push_back(buf + off[i]);
    w.K.push_back(buf + off[i] + n2);
  }
  fock_status s = tune(w, b, reps, tuned, ms, pair_ms);
  cudaStreamSynchronize(stream);
  cudaFree(buf);
  return s;
}
