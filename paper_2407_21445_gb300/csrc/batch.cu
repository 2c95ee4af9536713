// fock_build_jk_batched: many molecules in one pass.
//
// The shell-pair data of every molecule are merged into one device set
// (shell, pair and primitive indices offset per molecule; basis-function
// indices stay molecule-local) and their work units into one unit list per
// class tier, so that one launch per tier covers all molecules.  D, J and K
// stay separate caller buffers per molecule, reached through a per-molecule
// table.  The whole sequence (table upload, zeroing, density preparation,
// every tier, symmetrisation) is captured once into a CUDA graph on a
// private stream and replayed on later calls with the same molecules and
// threshold; merged plans are cached per list of handles.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "fock_impl.h"

namespace fk {
fock_status upload_staging(const Staging &st, const std::vector<Unit> &units, void **base, DevPairs &dp,
                           Unit **d_units, size_t *bytes, cudaStream_t stream);
}

using namespace fk;

namespace {

struct BatchPlan {
  std::vector<unsigned long long> key;
  int device = 0, nmol = 0;
  bool mixed = false;
  double cutoff = 0.0;
  double prim_eps = 0.0;  // primitive-quartet screening factor (prune_eps)
  DevPairs dev{};
  void *d_block = nullptr;
  std::vector<Tier> tiers;
  std::vector<MolEntry> stat;         // static fields per molecule
  long long dsh_total = 0, n2_total = 0;
  void *d_aux = nullptr;              // table, prefixes, scratch (one allocation)
  MolEntry *d_mt = nullptr;
  long long *d_dshp = nullptr, *d_n2p = nullptr;
  double *Dsh = nullptr;
  float *Dshf = nullptr, *Df = nullptr;
  int *counters = nullptr;
  MolEntry *h_mt = nullptr;           // pinned staging of the per-call table
  cudaStream_t st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_table = nullptr;
  bool table_pending = false;
  cudaGraphExec_t gexec = nullptr;
  double graph_tau = -1.0;

  ~BatchPlan() {
    if (st) cudaStreamSynchronize(st);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (d_block) cudaFree(d_block);
    if (d_aux) cudaFree(d_aux);
    if (h_mt) cudaFreeHost(h_mt);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (ev_table) cudaEventDestroy(ev_table);
    if (st) cudaStreamDestroy(st);
  }
};

std::mutex g_mu;
std::vector<BatchPlan *> g_plans;  // most recent last
constexpr size_t kMaxPlans = 4;

fock_status batch_status(cudaError_t e) { return cuda_status(e, "fock_build_jk_batched"); }

bool same_opts(const fock_shellpairs *a, const fock_shellpairs *b) {
  return a->tau_build == b->tau_build && a->opts.precision == b->opts.precision &&
         a->opts.fp32_cutoff == b->opts.fp32_cutoff && a->opts.prune_eps == b->opts.prune_eps &&
         a->opts.group_override == b->opts.group_override && a->opts.warp_scratch == b->opts.warp_scratch &&
         a->opts.reg_max_L == b->opts.reg_max_L && a->opts.tune_isolate == b->opts.tune_isolate &&
         memcmp(a->opts.schedule, b->opts.schedule, sizeof(a->opts.schedule)) == 0 && a->device == b->device;
}

fock_status build_plan(const fock_shellpairs *const *bases, int nmol, BatchPlan **out) {
  BatchPlan *bp = new BatchPlan();
  bp->nmol = nmol;
  bp->device = bases[0]->device;
  bp->mixed = bases[0]->opts.precision == FOCK_MIXED && bases[0]->opts.fp32_cutoff > 0.0;
  bp->cutoff = bases[0]->opts.fp32_cutoff;
  bp->prim_eps = bases[0]->prune_eps;
  Staging m;
  struct Key {
    int cb, ck, G, sb, tag;
    bool operator<(const Key &o) const {
      if (tag != o.tag) return tag < o.tag;
      if (cb != o.cb) return cb < o.cb;
      if (ck != o.ck) return ck < o.ck;
      if (G != o.G) return G < o.G;
      return sb < o.sb;
    }
  };
  std::map<Key, int> tier_of;
  std::vector<std::vector<Unit>> tier_units;
  long long shells = 0, pairs = 0, prims = 0, evals = 0;
  for (int i = 0; i < nmol; ++i) {
    const fock_shellpairs *sp = bases[i];
    const Staging &h = sp->host;
    bp->key.push_back(sp->serial);
    MolEntry e{};
    e.N = sp->nbf;
    e.s0 = (int)shells;
    e.ns = sp->nshell;
    e.dsh_off = bp->dsh_total;
    e.n2_off = bp->n2_total;
    bp->dsh_total += (long long)sp->nshell * sp->nshell;
    bp->n2_total += (long long)sp->nbf * sp->nbf;
    bp->stat.push_back(e);
    m.sxyz.insert(m.sxyz.end(), h.sxyz.begin(), h.sxyz.end());
    m.shl.insert(m.shl.end(), h.shl.begin(), h.shl.end());
    m.sbf.insert(m.sbf.end(), h.sbf.begin(), h.sbf.end());
    m.sl.insert(m.sl.end(), h.sl.begin(), h.sl.end());
    m.smol.insert(m.smol.end(), h.sl.size(), i);
    for (const int2 &ab : h.ab) m.ab.push_back(make_int2(ab.x + (int)shells, ab.y + (int)shells));
    m.G.insert(m.G.end(), h.G.begin(), h.G.end());
    m.Gf.insert(m.Gf.end(), h.Gf.begin(), h.Gf.end());
    m.cls.insert(m.cls.end(), h.cls.begin(), h.cls.end());
    for (const int2 &p : h.prim) m.prim.push_back(make_int2(p.x + (int)prims, p.y));
    m.pz.insert(m.pz.end(), h.pz.begin(), h.pz.end());
    m.pf.insert(m.pf.end(), h.pf.begin(), h.pf.end());
    m.paf.insert(m.paf.end(), h.paf.begin(), h.paf.end());
    m.U.insert(m.U.end(), h.U.begin(), h.U.end());
    m.Gp.insert(m.Gp.end(), h.Gp.begin(), h.Gp.end());
    m.Gpf.insert(m.Gpf.end(), h.Gpf.begin(), h.Gpf.end());
    m.Uf.insert(m.Uf.end(), h.Uf.begin(), h.Uf.end());
    for (int o : h.eoff) m.eoff.push_back(o + (int)evals);
    m.E.insert(m.E.end(), h.E.begin(), h.E.end());
    m.Ef.insert(m.Ef.end(), h.Ef.begin(), h.Ef.end());
    for (size_t u = 0; u < sp->h_units.size(); ++u) {
      const Tier &t = sp->tiers[sp->h_unit_tier[u]];
      const Key k{t.reg_cb, t.reg_ck, t.reg_cb >= 0 ? 0 : t.G, t.reg_cb >= 0 ? 0 : t.sb, t.tag};
      auto it = tier_of.find(k);
      int ti;
      if (it == tier_of.end()) {
        ti = (int)bp->tiers.size();
        tier_of[k] = ti;
        Tier nt = t;
        nt.nunits = 0;
        nt.d_units = nullptr;
        bp->tiers.push_back(nt);
        tier_units.emplace_back();
      } else {
        ti = it->second;
        bp->tiers[ti].stride = std::max(bp->tiers[ti].stride, t.stride);
      }
      Unit un = sp->h_units[u];
      un.bra += (int)pairs;
      un.k0 += (int)pairs;
      un.k1 += (int)pairs;
      tier_units[ti].push_back(un);
    }
    shells += sp->nshell;
    pairs += (long long)h.ab.size();
    prims += (long long)h.pz.size();
    evals += (long long)h.E.size();
  }
  if (shells > 0x7fffffffLL || evals > 0x7fffffffLL) {
    delete bp;
    return FOCK_ERR_INVALID_ARG;
  }
  std::vector<Unit> all;
  std::vector<size_t> first;
  for (size_t t = 0; t < bp->tiers.size(); ++t) {
    first.push_back(all.size());
    all.insert(all.end(), tier_units[t].begin(), tier_units[t].end());
    bp->tiers[t].nunits = (int)tier_units[t].size();
  }
  cudaError_t ce = cudaStreamCreateWithFlags(&bp->st, cudaStreamNonBlocking);
  if (ce != cudaSuccess) {
    delete bp;
    return batch_status(ce);
  }
  Unit *d_units = nullptr;
  fock_status s = upload_staging(m, all, &bp->d_block, bp->dev, &d_units, nullptr, bp->st);
  if (s != FOCK_OK) {
    delete bp;
    return s;
  }
  bp->dev.nshell = (int)shells;
  bp->dev.nbf = 0;  // per molecule, from the table
  for (size_t t = 0; t < bp->tiers.size(); ++t) {
    bp->tiers[t].d_units = d_units + first[t];
    ce = configure_tier(bp->tiers[t]);
    if (ce != cudaSuccess) {
      delete bp;
      return batch_status(ce);
    }
  }
  // table, prefixes and scratch in one allocation
  const size_t nt = bp->tiers.size();
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t off = 0;
  const size_t o_mt = off;
  off = al(off + sizeof(MolEntry) * nmol);
  const size_t o_dshp = off;
  off = al(off + sizeof(long long) * (nmol + 1));
  const size_t o_n2p = off;
  off = al(off + sizeof(long long) * (nmol + 1));
  const size_t o_dsh = off;
  off = al(off + sizeof(double) * bp->dsh_total);
  const size_t o_dshf = off;
  off = al(off + sizeof(float) * bp->dsh_total);
  const size_t o_cnt = off;
  off = al(off + sizeof(int) * (2 * nt + 1));
  const size_t o_df = off;
  if (bp->mixed) off = al(off + sizeof(float) * bp->n2_total);
  char *aux = nullptr;
  ce = cudaMalloc(&aux, off);
  if (ce != cudaSuccess) {
    delete bp;
    return batch_status(ce);
  }
  bp->d_aux = aux;
  bp->d_mt = (MolEntry *)(aux + o_mt);
  bp->d_dshp = (long long *)(aux + o_dshp);
  bp->d_n2p = (long long *)(aux + o_n2p);
  bp->Dsh = (double *)(aux + o_dsh);
  bp->Dshf = (float *)(aux + o_dshf);
  bp->counters = (int *)(aux + o_cnt);
  bp->Df = bp->mixed ? (float *)(aux + o_df) : nullptr;
  std::vector<long long> dshp(nmol + 1), n2p(nmol + 1);
  for (int i = 0; i < nmol; ++i) {
    dshp[i] = bp->stat[i].dsh_off;
    n2p[i] = bp->stat[i].n2_off;
  }
  dshp[nmol] = bp->dsh_total;
  n2p[nmol] = bp->n2_total;
  ce = cudaMemcpyAsync(bp->d_dshp, dshp.data(), sizeof(long long) * (nmol + 1), cudaMemcpyHostToDevice, bp->st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(bp->d_n2p, n2p.data(), sizeof(long long) * (nmol + 1), cudaMemcpyHostToDevice, bp->st);
  if (ce == cudaSuccess) ce = cudaMallocHost(&bp->h_mt, sizeof(MolEntry) * nmol);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&bp->ev_in, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&bp->ev_out, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&bp->ev_table, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(bp->st);
  if (ce != cudaSuccess) {
    delete bp;
    return batch_status(ce);
  }
  *out = bp;
  return FOCK_OK;
}

// ev (optional, tiers + 1 events): recorded before every tier and after the last.
cudaError_t enqueue(BatchPlan *bp, double tau, const cudaEvent_t *ev = nullptr) {
  cudaStream_t st = bp->st;
  cudaError_t e = cudaMemcpyAsync(bp->d_mt, bp->h_mt, sizeof(MolEntry) * bp->nmol, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bp->counters, 0, sizeof(int) * (2 * bp->tiers.size() + 1), st);
  if (e == cudaSuccess) e = launch_zero_batch(bp->d_mt, bp->d_n2p, bp->nmol, bp->n2_total, st);
  if (e == cudaSuccess)
    e = launch_dprep_batch(bp->d_mt, bp->d_dshp, bp->nmol, bp->dsh_total, bp->dev.sbf, bp->dev.sl, bp->Dsh,
                           bp->Dshf, st);
  for (size_t t = 0; t < bp->tiers.size() && e == cudaSuccess; ++t) {
    if (ev) e = cudaEventRecord(ev[t], st);
    if (e == cudaSuccess)
      e = launch_jk_tier_batch(bp->tiers[t], bp->dev, bp->d_mt, bp->Dsh, bp->Dshf, tau, bp->prim_eps,
                               bp->counters + t, bp->counters + bp->tiers.size() + t, st,
                               bp->mixed ? bp->cutoff : 0.0);
  }
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[bp->tiers.size()], st);
  if (e == cudaSuccess) e = launch_symmetrize_batch(bp->d_mt, bp->d_n2p, bp->nmol, bp->n2_total, st);
  return e;
}

}  // namespace

namespace fk {
// The batched build of `bases` run `reps` times from a fresh merged plan,
// without a graph, with events around every tier: ms_by_tag[tag] receives,
// per tier tag, the smallest over the runs of the summed tier times
// (class-pair timing for fock_autotune).  Synchronous.
fock_status batch_tier_times(const fock_shellpairs *const *bases, int nmol, const double *const *D, double tau,
                             double *const *J, double *const *K, int reps, cudaStream_t stream,
                             std::vector<double> &ms_by_tag) {
  std::lock_guard<std::mutex> lk(g_mu);
  BatchPlan *bp = nullptr;
  fock_status s = build_plan(bases, nmol, &bp);
  if (s != FOCK_OK) return s;
  const size_t nt = bp->tiers.size();
  std::vector<cudaEvent_t> ev(nt + 1, nullptr);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i <= nt && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  for (int i = 0; i < nmol; ++i) {
    MolEntry m = bp->stat[i];
    m.D = D[i];
    m.J = J[i];
    m.K = K[i];
    m.Df = bp->mixed ? bp->Df + m.n2_off : nullptr;
    bp->h_mt[i] = m;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  std::vector<double> best;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // run 0 warms up
    e = enqueue(bp, tau, ev.data());
    if (e == cudaSuccess) e = cudaStreamSynchronize(bp->st);
    if (e != cudaSuccess || r == 0) continue;
    std::vector<double> cur(ms_by_tag.size(), 0.0);
    for (size_t t = 0; t < nt && e == cudaSuccess; ++t) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[t], ev[t + 1]);
      const int tag = bp->tiers[t].tag;
      if (tag >= 0 && tag < (int)cur.size()) cur[tag] += ms;
    }
    if (best.empty()) best = cur;
    for (size_t i = 0; i < cur.size(); ++i) best[i] = std::min(best[i], cur[i]);
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  delete bp;
  if (e != cudaSuccess) return batch_status(e);
  for (size_t i = 0; i < best.size(); ++i) ms_by_tag[i] = best[i];
  return FOCK_OK;
}
}  // namespace fk

extern "C" fock_status fock_build_jk_batched(const fock_shellpairs *const *bases, int32_t nmol,
                                             const double *const *D, double schwarz_thresh, double *const *J,
                                             double *const *K, cudaStream_t stream) {
  if (!bases || nmol < 0 || !D || !J || !K) return FOCK_ERR_INVALID_ARG;
  if (nmol == 0) return FOCK_OK;
  for (int i = 0; i < nmol; ++i) {
    if (!bases[i] || !D[i] || !J[i] || !K[i]) return FOCK_ERR_INVALID_ARG;
    if (!same_opts(bases[0], bases[i])) return FOCK_ERR_INVALID_ARG;
    if (bases[i]->opts.k_mode != FOCK_K_EXACT) return FOCK_ERR_INVALID_ARG;  // exact exchange test only
  }
  if (!(schwarz_thresh >= bases[0]->tau_build) || !isfinite(schwarz_thresh)) return FOCK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  BatchPlan *bp = nullptr;
  for (BatchPlan *p : g_plans) {
    if ((int)p->key.size() != nmol) continue;
    bool same = true;
    for (int i = 0; i < nmol && same; ++i) same = p->key[i] == bases[i]->serial;
    if (same) {
      bp = p;
      break;
    }
  }
  if (!bp) {
    fock_status s = build_plan(bases, nmol, &bp);
    if (s != FOCK_OK) return s;
    if (g_plans.size() >= kMaxPlans) {
      delete g_plans.front();
      g_plans.erase(g_plans.begin());
    }
    g_plans.push_back(bp);
  }
  // the pinned table may still be read by the previous replay
  cudaError_t e = cudaSuccess;
  if (bp->table_pending) e = cudaEventSynchronize(bp->ev_table);
  if (e != cudaSuccess) return batch_status(e);
  for (int i = 0; i < nmol; ++i) {
    MolEntry m = bp->stat[i];
    m.D = D[i];
    m.J = J[i];
    m.K = K[i];
    m.Df = bp->mixed ? bp->Df + m.n2_off : nullptr;
    bp->h_mt[i] = m;
  }
  e = cudaEventRecord(bp->ev_in, stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(bp->st, bp->ev_in, 0);
  if (e != cudaSuccess) return batch_status(e);
  if (!bp->gexec || bp->graph_tau != schwarz_thresh) {
    if (bp->gexec) {
      cudaGraphExecDestroy(bp->gexec);
      bp->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(bp->st, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t ee = enqueue(bp, schwarz_thresh);
      e = cudaStreamEndCapture(bp->st, &g);
      if (ee != cudaSuccess) e = ee;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bp->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      bp->gexec = nullptr;
      return batch_status(e);
    }
    bp->graph_tau = schwarz_thresh;
  }
  e = cudaGraphLaunch(bp->gexec, bp->st);
  if (e == cudaSuccess) e = cudaEventRecord(bp->ev_table, bp->st);
  bp->table_pending = e == cudaSuccess;
  if (e == cudaSuccess) e = cudaEventRecord(bp->ev_out, bp->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, bp->ev_out, 0);
  return batch_status(e);
}
