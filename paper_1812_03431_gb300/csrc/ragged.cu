// Ragged batches: states of several plans (mixed truncations N and pole counts P)
// whose banded solves run as ONE persistent launch over the union of their work
// items, sorted longest first (the per-item plan index selects factors, layout and
// buffers).  Inputs are gathered into each plan's internal layout and results
// scattered back, up to 32 states per launch; after a first call with the same
// per-plan state counts nothing is allocated, so the step can be captured in a
// CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "rexi_internal.h"

struct rexi_plan {
  rexi::Plan *pl;
};

namespace rexi {
rexi_status get_layout(Plan &pl, int B, bool single, SolveLayout **out);
}

struct rexi_ragged {
  std::vector<rexi::Plan *> plans;
  int max_states = 0, lmax = 1, resident_warps = 0;
  double2 *ybuf = nullptr;
  unsigned *counter = nullptr;
  struct Cfg {
    rexi::SolveView *views_dev = nullptr;
    rexi::WorkItem *items_dev = nullptr;
    int nitems = 0;
    std::vector<uint64_t> gens;  // the plans' layout generations the views were built from
    bool fused = false;          // binary64 plans: the fused solve over every plan's items
    rexi::FusedRagged fr;
  };
  std::map<std::vector<int>, Cfg> cfgs;
};

namespace rexi {
namespace {

// s_int[(f * nspec + idx) * B + b] <-> state[f * nspec + idx], for up to kMoveChunk states
// per launch (blockIdx.y), their pointers passed by value so that a captured graph keeps them
constexpr int kMoveChunk = 32;
struct StateMoves {
  const double2 *src[kMoveChunk];
  double2 *dst[kMoveChunk];
  int64_t n3[kMoveChunk];
  int B[kMoveChunk], b[kMoveChunk];
};
template <bool kGather>
__global__ void move_states_kernel(StateMoves m) {
  const int s = blockIdx.y;
  const int64_t n3 = m.n3[s];
  const int B = m.B[s], b = m.b[s];
  const double2 *src = m.src[s];
  double2 *dst = m.dst[s];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += (int64_t)gridDim.x * blockDim.x) {
    if (kGather) dst[t * B + b] = src[t];
    else dst[t] = src[t * B + b];
  }
}

// every state into (gather) or out of (scatter) its plan's internal layout, in launches of
// up to kMoveChunk states
cudaError_t move_states(const std::vector<Plan *> &plans, const void *const *ext, const int32_t *state_plan,
                        int nstates, const std::vector<int> &counts, const std::vector<int> &rank, bool gather,
                        cudaStream_t st) {
  for (int s0 = 0; s0 < nstates; s0 += kMoveChunk) {
    const int n = std::min(kMoveChunk, nstates - s0);
    StateMoves m{};
    int64_t n3max = 1;
    for (int i = 0; i < n; ++i) {
      const int s = s0 + i, p = state_plan[s];
      Plan &pl = *plans[p];
      m.n3[i] = 3 * pl.nspec;
      m.B[i] = counts[p];
      m.b[i] = rank[s];
      m.src[i] = gather ? static_cast<const double2 *>(ext[s]) : pl.s_out;
      m.dst[i] = gather ? pl.s_in : static_cast<double2 *>(const_cast<void *>(ext[s]));
      n3max = std::max(n3max, m.n3[i]);
    }
    const dim3 grid((unsigned)std::min<int64_t>((n3max + 255) / 256, 512), (unsigned)n);
    if (gather) move_states_kernel<true><<<grid, 256, 0, st>>>(m);
    else move_states_kernel<false><<<grid, 256, 0, st>>>(m);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

rexi_status fail(const std::string &what, cudaError_t e) {
  set_error("ragged: " + what + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? REXI_ENOMEM : REXI_ECUDA;
}

}  // namespace
}  // namespace rexi

using namespace rexi;

extern "C" {

rexi_status rexi_ragged_create(rexi_plan *const *plans, int32_t nplans, int32_t max_states, rexi_ragged **out) {
  if (!out || !plans || nplans < 1 || max_states < 1) {
    set_error("rexi_ragged_create: need plans, nplans >= 1, max_states >= 1");
    return REXI_EINVAL;
  }
  *out = nullptr;
  rexi_ragged *rg = new rexi_ragged();
  rg->max_states = max_states;
  for (int i = 0; i < nplans; ++i) {
    if (!plans[i] || !plans[i]->pl || plans[i]->pl->prm.layout != REXI_SPECTRAL || plans[i]->pl->prm.fsphere ||
        plans[i]->pl->prm.solver != REXI_SOLVER_DELTA) {
      delete rg;
      set_error("rexi_ragged_create: every plan must exist, use REXI_SPECTRAL, the rotating sphere and "
                "REXI_SOLVER_DELTA");
      return REXI_EINVAL;
    }
    if (plans[i]->pl->ff != plans[0]->pl->ff) {
      delete rg;
      set_error("rexi_ragged_create: every plan must use the same solve_arith");
      return REXI_EINVAL;
    }
    rg->plans.push_back(plans[i]->pl);
    rg->lmax = std::max(rg->lmax, plans[i]->pl->lmax);
    rg->resident_warps = std::max(rg->resident_warps, plans[i]->pl->resident_warps);
  }
  cudaError_t e = cudaMalloc(&rg->ybuf, (size_t)rg->resident_warps * rg->lmax * sweep_width(rg->plans[0]->ff) * 32 *
                                            sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&rg->counter, sizeof(unsigned));
  if (e != cudaSuccess) {
    rexi_ragged_destroy(rg);
    return fail("allocation", e);
  }
  *out = rg;
  return REXI_OK;
}

rexi_status rexi_ragged_step(rexi_ragged *rg, const void *const *in_dev, void *const *out_dev,
                             const int32_t *state_plan, int32_t nstates, void *stream) {
  if (!rg || !in_dev || !out_dev || !state_plan || nstates < 1 || nstates > rg->max_states) {
    set_error("rexi_ragged_step: bad arguments or nstates > max_states");
    return REXI_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int np = (int)rg->plans.size();
  std::vector<int> counts(np, 0), rank(nstates);
  for (int s = 0; s < nstates; ++s) {
    const int p = state_plan[s];
    if (p < 0 || p >= np || !in_dev[s] || !out_dev[s]) {
      set_error("rexi_ragged_step: state " + std::to_string(s) + " has a bad plan index or pointer");
      return REXI_EINVAL;
    }
    rank[s] = counts[p]++;
  }
  for (int p = 0; p < np; ++p)
    if (counts[p] > rg->plans[p]->prm.max_batch) {
      set_error("rexi_ragged_step: more states for plan " + std::to_string(p) + " than its max_batch");
      return REXI_EINVAL;
    }
  // binary64 plans: one fused launch over every plan's items (the pole sum on chip, no
  // reductions); else the slot kernel over the merged work list, then per-plan reductions.
  // Either work list is cached per count vector.
  auto it = rg->cfgs.find(counts);
  if (it == rg->cfgs.end() && !rg->plans[0]->ff) {
    rexi_ragged::Cfg cfg;
    if (build_fused_ragged(rg->plans, counts, cfg.fr)) {
      cfg.fused = true;
      it = rg->cfgs.emplace(counts, cfg).first;
    }
  }
  const bool fused = it != rg->cfgs.end() && it->second.fused;
  std::vector<SolveLayout *> lays(np, nullptr);
  for (int p = 0; p < np && !fused; ++p)
    if (counts[p] > 0) {
      rexi_status r = get_layout(*rg->plans[p], counts[p], false, &lays[p]);
      if (r != REXI_OK) return r;
    }
  std::vector<uint64_t> gens(np);
  for (int p = 0; p < np; ++p) gens[p] = rg->plans[p]->layout_gen;
  if (!fused && it != rg->cfgs.end() && it->second.gens != gens) {
    // a plan's slot layout was replaced (rexi_tune, rexi_set_pole_slots) since this work
    // list was built: its views point at the freed one, so it is rebuilt.  No step of
    // this ragged object may be in flight meanwhile (the same rule as for the tuning call)
    if (it->second.views_dev) cudaFree(it->second.views_dev);
    if (it->second.items_dev) cudaFree(it->second.items_dev);
    rg->cfgs.erase(it);
    it = rg->cfgs.end();
  }
  if (it == rg->cfgs.end()) {
    std::vector<SolveView> views(np);
    struct Tagged { WorkItem w; double work; };
    std::vector<Tagged> all;
    for (int p = 0; p < np; ++p) {
      if (counts[p] == 0) continue;
      Plan &pl = *rg->plans[p];
      const SolveLayout &L = *lays[p];
      views[p] = make_view(pl, L, false, pl.ff ? pl.s_ff : pl.s_in, pl.partial, counts[p], 0, pl.P);
      const int nb = (counts[p] + L.bw - 1) / L.bw;
      for (int m = 0; m <= pl.N; ++m) {
        const int l = std::max(pl.sys[2 * m].len, pl.sys[2 * m + 1].len);
        if (l == 0) continue;
        const int sm = L.groups_m[m] * L.kk;
        const double work = (double)l * ((pl.P + sm - 1) / sm);
        for (int g = 0; g < L.groups_m[m]; ++g)
          for (int bb = 0; bb < nb; ++bb) all.push_back(Tagged{WorkItem{m, g, bb * L.bw, p}, work});
      }
    }
    std::stable_sort(all.begin(), all.end(), [](const Tagged &x, const Tagged &y) { return x.work > y.work; });
    std::vector<WorkItem> items;
    for (const Tagged &t : all) items.push_back(t.w);
    rexi_ragged::Cfg cfg;
    cfg.nitems = (int)items.size();
    cfg.gens = gens;
    cudaError_t e = cudaMalloc(&cfg.views_dev, views.size() * sizeof(SolveView));
    if (e == cudaSuccess) e = cudaMalloc(&cfg.items_dev, std::max<size_t>(1, items.size()) * sizeof(WorkItem));
    if (e == cudaSuccess) e = cudaMemcpy(cfg.views_dev, views.data(), views.size() * sizeof(SolveView), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cfg.items_dev, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail("work list", e);
    it = rg->cfgs.emplace(counts, cfg).first;
  }
  const rexi_ragged::Cfg &cfg = it->second;
  cudaError_t e = move_states(rg->plans, in_dev, state_plan, nstates, counts, rank, true, st);
  const bool ff = rg->plans[0]->ff;
  if (cfg.fused) {
    if (e == cudaSuccess) e = launch_fused_ragged(cfg.fr, rg->ybuf, rg->plans[0]->num_sms, st);
  } else {
    for (int p = 0; p < np && e == cudaSuccess; ++p)  // float-float solves read split states
      if (ff && counts[p] > 0) {
        Plan &pl = *rg->plans[p];
        e = launch_split_state(pl, pl.s_in, pl.s_ff, 3 * pl.nspec * counts[p], st);
      }
    if (e == cudaSuccess)
      e = launch_solve_ragged(cfg.views_dev, cfg.items_dev, cfg.nitems, rg->ybuf, rg->lmax, rg->counter,
                              rg->resident_warps, ff, st);
    for (int p = 0; p < np && e == cudaSuccess; ++p)
      if (counts[p] > 0)
        e = launch_reduce(*rg->plans[p], *lays[p], false, rg->plans[p]->s_in, rg->plans[p]->s_out, counts[p],
                          false, 0, st);
  }
  if (e == cudaSuccess)
    e = move_states(rg->plans, reinterpret_cast<const void *const *>(out_dev), state_plan, nstates, counts, rank,
                    false, st);
  return e == cudaSuccess ? REXI_OK : fail("launch", e);
}

void rexi_ragged_destroy(rexi_ragged *rg) {
  if (!rg) return;
  for (auto &kv : rg->cfgs) {
    if (kv.second.views_dev) cudaFree(kv.second.views_dev);
    if (kv.second.items_dev) cudaFree(kv.second.items_dev);
    free_fused_ragged(kv.second.fr);
  }
  if (rg->ybuf) cudaFree(rg->ybuf);
  if (rg->counter) cudaFree(rg->counter);
  delete rg;
}

}  // extern "C"
