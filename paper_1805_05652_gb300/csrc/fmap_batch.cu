// Uneven batches: many independent F-map instances (each its own atoms, grid,
// window and template count) run by one captured CUDA graph.
//
// Every instance gets a plan carved out of one batch workspace: rectangular
// windows take the FP64 prefix path, exponential windows the decayed-suffix
// recurrence (FP64-class accuracy).  The single-plan pipeline -- input
// checks, index tables, antenna sums and 2F coefficients, data sums and
// cells, fix-up of ill-conditioned cells, reductions -- runs phase by
// phase, and each phase is ONE persistent launch over the work units of all
// instances (fmap_batch.cuh): a grid of (SMs x occupancy) blocks pulls units
// from an atomic counter, heaviest instances first, and runs the same device
// bodies as the single-plan kernels.  Instances are grouped into waves whose
// workspace fits the memory budget; every wave's counter resets and phase
// launches are captured once into a CUDA graph that fmap_batch_run replays.
//
// Autotuning (FMAP_BATCH_AUTOTUNE): the occupancy of each phase's persistent
// launch and the templates per block of the recurrence are chosen by timing
// the candidates on the batch itself, per size class of the batch (a
// signature of its shape); choices are cached in memory for later batches of
// the same class.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "fmap_batch.cuh"

namespace fmap {

namespace {

constexpr int kOccCandidates[] = {1, 2, 4, 8};

struct Tuning {
  int occ[BP_COUNT];
  int rec_tpb;   // templates per block of the recurrence phase
};

std::mutex g_tune_mu;
std::map<std::string, Tuning> g_tune_cache;

// lanes: the scan width of the wave's exp instances (batch_scan_lanes).
const void* phase_kernel(int ph, int lanes) {
  if (const void* k = batch_kernel_common(ph)) return k;
  if (const void* k = batch_kernel_rect(ph)) return k;
  if (const void* k = batch_kernel_exp(ph, lanes)) return k;
  if (const void* k = batch_kernel_exp_rec(ph, lanes)) return k;
  return batch_kernel_fixup(ph);
}

int phase_threads(int ph, int lanes) {
  switch (ph) {
    case BP_FLAG_COUNT:
    case BP_FLAG_SCAN:
    case BP_FLAG_WRITE: return 1024;
    case BP_FIXUP: return 128;
    case BP_EXP_ANT:
    case BP_EXP_REC: return lanes;
    default: return 256;
  }
}

}  // namespace

struct Wave {
  std::vector<int32_t> items;            // instance indices (heaviest first)
  int lanes = kScanLanes;                // scan width of its exp instances
  BItem* d_items = nullptr;
  int64_t* d_offsets = nullptr;          // [BP_COUNT][n + 1]
  std::vector<int64_t> totals;           // units per phase
  size_t dyn_smem[BP_COUNT] = {};
};

}  // namespace fmap

struct fmap_batch_s {
  int device = 0, n_sm = 0;
  std::vector<fmap_batch_item> items;
  std::vector<fmap_plan_s*> plans;
  std::vector<double> cost;
  std::vector<fmap::Wave> waves;
  char* ws = nullptr;                    // instance workspaces of the largest wave
  size_t ws_bytes = 0;
  unsigned long long* d_counters = nullptr;   // [waves][BP_COUNT]
  uint32_t* d_err = nullptr;             // shared device status word
  fmap::Tuning tune{};
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t n_launches = 0;
};

namespace fmap {

static fmap_status batch_fail(const std::string& m, fmap_status st = FMAP_ERR_ARG) {
  set_error(m);
  return st;
}

// Work units of instance `p` in phase `ph` (0: phase not used by it).
static int64_t units_of(const fmap_plan_s* p, const fmap_batch_item& it, int ph, int rec_tpb) {
  const fmap_grid& g = p->grid;
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const int64_t T = p->n_templates;
  const int64_t n_ant = it.atoms.shared_antenna ? 1 : T;
  const bool rect = g.window == FMAP_RECT;
  const bool work = cells > 0 && T > 0;
  switch (ph) {
    case BP_PREP:   // relative times, then the clearing of the marked-entry bitmask
      return (p->n_sft > 0 ? (rel_t_entries(p->n_sft) + 255) / 256 : 0) +
             (work ? (flag_words(cells * n_ant) + kBitsPerUnit - 1) / kBitsPerUnit : 0);
    case BP_INDEX: return cells > 0 ? (g.n_t0 + kIdxRowsPerUnit - 1) / kIdxRowsPerUnit : 0;
    case BP_EXP_PERM: {
      if (rect || cells == 0) return 0;
      const int32_t n_x = (p->flags & FMAP_PLAN_EXP_RECURRENCE) ? (int32_t)T : 0;
      return (exp_copy_entries(p->n_sft, p->lanes, (int32_t)n_ant, n_x, g.n_tau) + kPermPerUnit - 1) /
             kPermPerUnit;
    }
    case BP_RECT_ANT: return rect && cells > 0 && p->n_sft > 0 ? n_ant : 0;
    case BP_EXP_ANT: return !rect && cells > 0 ? g.n_tau * n_ant : 0;
    case BP_RECT_COEF:
      return rect && cells > 0 ? (cells * n_ant + 256 * kCoefBlocksPerUnit - 1) / (256 * kCoefBlocksPerUnit) : 0;
    case BP_RECT_DATA: return rect && work && p->n_sft > 0 ? T : 0;
    case BP_EXP_REC: return !rect && work ? g.n_tau * ((T + rec_tpb - 1) / rec_tpb) : 0;
    case BP_RECT_CELLS:
      return rect && work ? rect_cells_blocks(g, (int32_t)T, it.atoms.shared_antenna) : 0;
    case BP_FLAG_COUNT:
    case BP_FLAG_WRITE: return work ? (cells * n_ant + kFlagUnit - 1) / kFlagUnit : 0;
    case BP_FLAG_SCAN: return work ? 1 : 0;
    case BP_FIXUP: return work ? (int64_t)(kFixSlots / kFixSlotsPerUnit) * fixup_blocks_y((int32_t)T) : 0;
    case BP_RED_GROUPS: {
      if (!it.d_summary || T == 0) return 0;
      const int64_t used =
          cells > 0 ? (rect ? rect_partial_slots(g, (int32_t)T, it.atoms.shared_antenna) : g.n_tau) : 0;
      return reduce_groups_of(used + (cells > 0 ? kFixSlots : 0)) * T;
    }
    case BP_RED_FINAL: return it.d_summary && T > 0 ? T : 0;
  }
  return 0;
}

static BItem make_bitem(const fmap_plan_s* p, const fmap_batch_item& it, uint32_t* err,
                        int rec_tpb) {
  BItem b{};
  const fmap_grid& g = p->grid;
  b.g = g;
  b.n_sft = p->n_sft;
  b.T = p->n_templates;
  b.shared = it.atoms.shared_antenna ? 1 : 0;
  b.n_ant = b.shared ? 1 : b.T;
  b.groups = std::max(1, (b.T + rec_tpb - 1) / rec_tpb);
  b.n_alloc = rel_t_entries(p->n_sft);
  b.lanes = p->lanes;
  b.cells = (int64_t)g.n_t0 * g.n_tau;
  b.n_tiles = p->n_tiles;
  b.part_stride = p->part_stride;
  b.tiles_used = b.cells > 0 ? (g.window == FMAP_RECT ? rect_partial_slots(g, b.T, b.shared) : g.n_tau) : 0;
  b.red_groups = reduce_groups_of(b.tiles_used + (b.cells > 0 ? kFixSlots : 0));
  b.flag_entries = b.cells * b.n_ant;
  b.log_prior = p->log_prior;
  b.t = it.atoms.t;
  b.antenna = it.atoms.antenna;
  b.fafb = it.atoms.fafb;
  b.map = it.d_2F;
  b.summary = it.d_summary;
  const Workspace& w = p->ws;
  b.rel_t = w.rel_t;
  b.t_base = w.t_base;
  b.dev_err = err;
  b.i0 = w.i0;
  b.jend = w.jend;
  b.coef = w.coef;
  b.partials = w.partials;
  b.red_buf = w.groups;
  b.flag_blocks = w.flag_blocks;
  b.flag_bits = w.flag_bits;
  b.n_flag = w.n_flag;
  b.flag_list = w.flag_list;
  b.pa = w.pa;
  b.perm_ant = w.perm_ant;
  b.perm_x = w.perm_x;
  b.perm_gap = w.perm_gap;
  b.rec_cells = w.rec_cells;
  b.tauc = w.tauc;
  b.ax = nullptr;   // batches take uniform grids
  b.px = w.px;
  return b;
}

// Upload one wave's instance table and unit offsets for a tuning choice.
static fmap_status build_wave_tables(fmap_batch_s* B, Wave& wv, const Tuning& tn) {
  const int n = (int)wv.items.size();
  std::vector<BItem> h(n);
  std::vector<int64_t> off((size_t)BP_COUNT * (n + 1), 0);
  wv.totals.assign(BP_COUNT, 0);
  for (int ph = 0; ph < BP_COUNT; ++ph) wv.dyn_smem[ph] = 0;
  for (int k = 0; k < n; ++k) {
    const int32_t i = wv.items[k];
    const fmap_plan_s* p = B->plans[i];
    h[k] = make_bitem(p, B->items[i], B->d_err, tn.rec_tpb);
    for (int ph = 0; ph < BP_COUNT; ++ph) {
      const int64_t u = units_of(p, B->items[i], ph, tn.rec_tpb);
      off[(size_t)ph * (n + 1) + k + 1] = off[(size_t)ph * (n + 1) + k] + u;
      if (u > 0) {
        if (ph == BP_EXP_ANT)
          wv.dyn_smem[ph] = std::max(wv.dyn_smem[ph], exp_antenna_smem(p->n_sft));
        if (ph == BP_EXP_REC)
          wv.dyn_smem[ph] = std::max(
              wv.dyn_smem[ph],
              exp_rec_smem(p->n_sft, p->grid.n_t0,
                           (h[k].T + h[k].groups - 1) / std::max(1, h[k].groups)));
        if (ph == BP_RECT_CELLS)
          wv.dyn_smem[ph] = std::max(wv.dyn_smem[ph], rect_cells_smem(p->n_templates, B->items[i].atoms.shared_antenna));
      }
    }
  }
  for (int ph = 0; ph < BP_COUNT; ++ph) wv.totals[ph] = off[(size_t)ph * (n + 1) + n];
  if (!wv.d_items) {
    FMAP_CUDA(cudaMalloc(&wv.d_items, sizeof(BItem) * std::max(n, 1)));
    FMAP_CUDA(cudaMalloc(&wv.d_offsets, sizeof(int64_t) * off.size()));
  }
  FMAP_CUDA(cudaMemcpy(wv.d_items, h.data(), sizeof(BItem) * n, cudaMemcpyHostToDevice));
  FMAP_CUDA(cudaMemcpy(wv.d_offsets, off.data(), sizeof(int64_t) * off.size(),
                       cudaMemcpyHostToDevice));
  return FMAP_OK;
}

// Enqueue one phase of one wave (counter reset + persistent launch).
static fmap_status enqueue_phase(fmap_batch_s* B, int w, int ph, int occ, cudaStream_t s) {
  Wave& wv = B->waves[w];
  const int64_t total = wv.totals[ph];
  if (total == 0) return FMAP_OK;
  const void* k = phase_kernel(ph, wv.lanes);
  const int threads = phase_threads(ph, wv.lanes);
  // narrower exp blocks: the same occupancy candidates in units of 256 threads
  if (ph == BP_EXP_ANT || ph == BP_EXP_REC) occ *= kScanLanes / wv.lanes;
  const size_t smem = wv.dyn_smem[ph];
  if (smem > 0)
    FMAP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int max_occ = 0;
  FMAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_occ, k, threads, smem));
  max_occ = std::max(1, max_occ);
  const int64_t grid = std::min<int64_t>(total, (int64_t)B->n_sm * std::min(occ, max_occ));
  unsigned long long* ctr = B->d_counters + (size_t)w * BP_COUNT + ph;
  FMAP_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s));
  BUnits u;
  u.offsets = wv.d_offsets + (size_t)ph * (wv.items.size() + 1);
  u.n_items = (int32_t)wv.items.size();
  u.total = total;
  u.counter = ctr;
  const BItem* items = wv.d_items;
  void* args[] = {(void*)&items, (void*)&u};
  FMAP_CUDA(cudaLaunchKernel(k, dim3((unsigned)grid), dim3(threads), args, smem, s));
  B->n_launches += 1;
  return FMAP_OK;
}

// Carve every instance's plan of wave w out of the shared workspace.
static fmap_status place_wave(fmap_batch_s* B, int w) {
  size_t off = 0;
  for (int32_t i : B->waves[w].items) {
    fmap_plan_s* p = B->plans[i];
    const fmap_batch_item& it = B->items[i];
    size_t bytes = 0;
    const uint32_t flags = (it.atoms.shared_antenna ? 0u : (uint32_t)FMAP_PLAN_PER_TEMPLATE_ANTENNA) |
                           (it.grid.window == FMAP_EXP ? (uint32_t)FMAP_PLAN_EXP_RECURRENCE : 0u) |
                           kPlanBatch;
    fmap_status st = plan_footprint(&it.grid, it.atoms.n_sft, it.atoms.n_templates, FMAP_FP64,
                                    flags, &bytes);
    if (st != FMAP_OK) return st;
    st = plan_init(p, &it.grid, it.atoms.n_sft, it.atoms.n_templates, FMAP_FP64, flags,
                   B->ws + off, bytes);
    if (st != FMAP_OK) return st;
    p->lanes = batch_scan_lanes(it.atoms.n_sft);   // the wave's exp kernels use this width
    off += (bytes + 255) / 256 * 256;
  }
  return FMAP_OK;
}

static std::string signature(const fmap_batch_s* B) {
  // size class: counts of instances per (window, log2 N_SFT, log2 cells, log2 T)
  std::map<std::string, int> h;
  for (size_t i = 0; i < B->items.size(); ++i) {
    const fmap_batch_item& it = B->items[i];
    const int64_t cells = (int64_t)it.grid.n_t0 * it.grid.n_tau;
    const std::string k = std::to_string(it.grid.window) + "/" +
                          std::to_string((int)std::log2(1.0 + it.atoms.n_sft)) + "/" +
                          std::to_string((int)std::log2(1.0 + cells)) + "/" +
                          std::to_string((int)std::log2(1.0 + it.atoms.n_templates));
    h[k] += 1;
  }
  std::string s;
  for (auto& kv : h) s += kv.first + ":" + std::to_string(kv.second) + ";";
  return s;
}

// Time each phase's candidates on the batch (single-wave batches; multi-wave
// batches use the occupancy the first wave prefers).
static fmap_status autotune(fmap_batch_s* B) {
  const std::string sig = signature(B);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      B->tune = it->second;
      return FMAP_OK;
    }
  }
  cudaStream_t s = B->cap;
  cudaEvent_t e0, e1;
  FMAP_CUDA(cudaEventCreate(&e0));
  FMAP_CUDA(cudaEventCreate(&e1));
  Tuning best = B->tune;
  fmap_status st = place_wave(B, 0);
  if (st == FMAP_OK) st = build_wave_tables(B, B->waves[0], best);
  // one full pass so every phase's inputs exist
  for (int ph = 0; st == FMAP_OK && ph < BP_COUNT; ++ph) st = enqueue_phase(B, 0, ph, best.occ[ph], s);
  for (int ph = 0; st == FMAP_OK && ph < BP_COUNT; ++ph) {
    if (B->waves[0].totals[ph] == 0) continue;
    // Candidates are timed by re-running one phase on the outputs of the full
    // pass; the compaction phases are not idempotent (the scan turns counts
    // into offsets in place), so they keep the default occupancy.
    if (ph == BP_FLAG_COUNT || ph == BP_FLAG_SCAN || ph == BP_FLAG_WRITE) continue;
    const bool rec = ph == BP_EXP_REC;
    const int tpbs[] = {1, 2, 4, 8};
    float best_ms = 1e30f;
    for (int ti = 0; ti < (rec ? 4 : 1) && st == FMAP_OK; ++ti) {
      Tuning tr = best;
      if (rec) {
        tr.rec_tpb = tpbs[ti];
        st = build_wave_tables(B, B->waves[0], tr);
      }
      for (int oc : kOccCandidates) {
        if (st != FMAP_OK) break;
        tr.occ[ph] = oc;
        // first run warms up; the fastest of the next three counts
        float ms = 1e30f;
        for (int rep = 0; rep < 4 && st == FMAP_OK; ++rep) {
          float r = 0.f;
          cudaEventRecord(e0, s);
          st = enqueue_phase(B, 0, ph, oc, s);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&r, e0, e1);
          if (rep > 0) ms = std::min(ms, r);
        }
        // a clearly faster candidate wins; within 5 % the higher occupancy
        // (the first wave is one size class, the others gain from parallelism)
        if (ms < 0.95f * best_ms || (ms <= 1.05f * best_ms && oc > best.occ[ph])) {
          best_ms = std::min(ms, best_ms);
          best.occ[ph] = oc;
          if (rec) best.rec_tpb = tr.rec_tpb;
        }
      }
    }
    if (rec && st == FMAP_OK) st = build_wave_tables(B, B->waves[0], best);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != FMAP_OK) return st;
  B->tune = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[sig] = best;
  return FMAP_OK;
}

static void batch_free(fmap_batch_s* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (auto& w : B->waves) {
    cudaFree(w.d_items);
    cudaFree(w.d_offsets);
  }
  for (auto* p : B->plans) {
    if (p) {
      plan_release(p);
      delete p;
    }
  }
  cudaFree(B->ws);
  cudaFree(B->d_counters);
  cudaFree(B->d_err);
  if (B->cap) cudaStreamDestroy(B->cap);
  delete B;
}

}  // namespace fmap

using namespace fmap;

static_assert(sizeof(fmap_batch_item) == 120, "fmap_batch_item layout");

extern "C" {

fmap_status fmap_batch_plan(fmap_batch_t** out, const fmap_batch_item* items, int32_t n_items,
                            size_t workspace_budget, uint32_t flags) {
  set_error("");
  if (!out || (!items && n_items > 0) || n_items < 0)
    return batch_fail("bad arguments");
  if (flags & ~(uint32_t)FMAP_BATCH_AUTOTUNE) return batch_fail("unknown batch flags");
  *out = nullptr;
  fmap_batch_s* B = new (std::nothrow) fmap_batch_s();
  if (!B) return FMAP_ERR_NOMEM;
  cudaGetDevice(&B->device);
  cudaDeviceGetAttribute(&B->n_sm, cudaDevAttrMultiProcessorCount, B->device);
  B->items.assign(items, items + n_items);
  B->plans.assign(n_items, nullptr);
  B->cost.assign(n_items, 0.0);
  std::vector<size_t> foot(n_items, 0);
  for (int32_t i = 0; i < n_items; ++i) {
    const fmap_batch_item& it = items[i];
    if (it.grid.window == FMAP_TABLE) {
      batch_free(B);
      return batch_fail("instance " + std::to_string(i) + ": table windows are not batched");
    }
    if (it.atoms.n_sft < 0 || it.atoms.n_templates < 0 ||
        (it.atoms.n_sft > 0 && (!it.atoms.t || !it.atoms.antenna ||
                                (it.atoms.n_templates > 0 && !it.atoms.fafb)))) {
      batch_free(B);
      return batch_fail("instance " + std::to_string(i) + ": bad atoms");
    }
    const uint32_t pf = (it.atoms.shared_antenna ? 0u : (uint32_t)FMAP_PLAN_PER_TEMPLATE_ANTENNA) |
                        (it.grid.window == FMAP_EXP ? (uint32_t)FMAP_PLAN_EXP_RECURRENCE : 0u) |
                        kPlanBatch;
    fmap_status st = plan_footprint(&it.grid, it.atoms.n_sft, it.atoms.n_templates, FMAP_FP64, pf,
                                    &foot[i]);
    if (st != FMAP_OK) {
      batch_free(B);
      set_error("instance " + std::to_string(i) + ": " + std::string(fmap_last_error()));
      return st;
    }
    foot[i] = (foot[i] + 255) / 256 * 256;
    B->plans[i] = new (std::nothrow) fmap_plan_s();
    // App. A cost model shape: c_SFT N_SFT + c_sums N_sums + c_F cells, per
    // template; the exp recurrence's sums scale like N_tau N_SFT.
    const double cells = (double)it.grid.n_t0 * it.grid.n_tau;
    const double sums = it.grid.window == FMAP_RECT ? cells
                                                    : (double)it.grid.n_tau * it.atoms.n_sft;
    B->cost[i] = (double)it.atoms.n_sft + (cells + sums) * std::max(1, it.atoms.n_templates);
  }
  // Shared-memory class of an instance: the exp phases launch with the
  // largest dynamic shared memory of their wave, so instances are grouped by
  // the number of blocks per SM that their exp kernels allow (rect instances
  // take the first class).  Within a class, heaviest first; waves are filled
  // greedily within the budget and never mix classes.  The class also
  // separates the exp scan widths (batch_scan_lanes), whose kernels differ.
  std::vector<int> cls(n_items, 0);
  auto lane_index = [](int32_t n) {
    return batch_scan_lanes(n) == 64 ? 0 : batch_scan_lanes(n) == 128 ? 1 : 2;
  };
  for (int32_t i = 0; i < n_items; ++i) {
    const fmap_batch_item& it = items[i];
    if (it.grid.window != FMAP_EXP) continue;
    const size_t sm = std::max(
        exp_rec_smem(it.atoms.n_sft, it.grid.n_t0, std::min(it.atoms.n_templates, 2)),
        exp_antenna_smem(it.atoms.n_sft));
    const int smem_cls = sm <= (56u << 10) ? 0 : sm <= (75u << 10) ? 1 : sm <= (113u << 10) ? 2 : 3;
    cls[i] = 4 * smem_cls + lane_index(it.atoms.n_sft);
  }
  std::vector<int32_t> order(n_items);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return cls[a] != cls[b] ? cls[a] < cls[b] : B->cost[a] > B->cost[b];
  });
  const size_t budget = workspace_budget ? workspace_budget : (size_t)8 << 30;
  size_t cur = 0, peak = 0;
  int cur_cls = -1;
  for (int32_t i : order) {
    if (foot[i] > budget) {
      batch_free(B);
      return batch_fail("instance " + std::to_string(i) + " alone exceeds the workspace budget",
                        FMAP_ERR_NOMEM);
    }
    if (B->waves.empty() || cur + foot[i] > budget || cls[i] != cur_cls) {
      B->waves.emplace_back();
      cur = 0;
      cur_cls = cls[i];
    }
    B->waves.back().items.push_back(i);
    if (items[i].grid.window == FMAP_EXP) B->waves.back().lanes = batch_scan_lanes(items[i].atoms.n_sft);
    cur += foot[i];
    peak = std::max(peak, cur);
  }
  cudaError_t e = cudaMalloc((void**)&B->ws, std::max<size_t>(peak, 256));
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&B->d_counters,
                   sizeof(unsigned long long) * BP_COUNT * std::max<size_t>(B->waves.size(), 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_err, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(B->d_err, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_free(B);
    return batch_fail("batch allocation failed", FMAP_ERR_NOMEM);
  }
  B->ws_bytes = peak;
  for (int ph = 0; ph < BP_COUNT; ++ph) B->tune.occ[ph] = 4;
  B->tune.rec_tpb = 1;
  fmap_status st = FMAP_OK;
  if ((flags & FMAP_BATCH_AUTOTUNE) && !B->waves.empty()) st = autotune(B);
  // Every wave's plans start at the workspace base: waves run one after the
  // other in the graph, so each reuses the memory of the previous one.
  for (size_t w = 0; w < B->waves.size() && st == FMAP_OK; ++w) {
    st = place_wave(B, (int)w);
    if (st == FMAP_OK) st = build_wave_tables(B, B->waves[w], B->tune);
  }
  if (st == FMAP_OK) {
    cudaStreamSynchronize(B->cap);
    B->n_launches = 0;
    e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCapture");
  }
  if (st == FMAP_OK) {
    for (size_t w = 0; w < B->waves.size() && st == FMAP_OK; ++w)
      for (int ph = 0; ph < BP_COUNT && st == FMAP_OK; ++ph)
        st = enqueue_phase(B, (int)w, ph, B->tune.occ[ph], B->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(B->cap, &g);
    if (st == FMAP_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture");
    B->graph = g;
    if (st == FMAP_OK) {
      e = cudaGraphInstantiate(&B->exec, g, 0);
      if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  if (st != FMAP_OK) {
    batch_free(B);
    return st;
  }
  *out = B;
  return FMAP_OK;
}

fmap_status fmap_batch_run(fmap_batch_t* B, fmap_stream stream) {
  set_error("");
  if (!B) return batch_fail("batch is NULL");
  FMAP_CUDA(cudaGraphLaunch(B->exec, (cudaStream_t)stream));
  return FMAP_OK;
}

fmap_status fmap_batch_status(fmap_batch_t* B, fmap_stream stream) {
  if (!B) return batch_fail("batch is NULL");
  FMAP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  uint32_t bits = 0;
  FMAP_CUDA(cudaMemcpy(&bits, B->d_err, sizeof(bits), cudaMemcpyDeviceToHost));
  if (bits) {
    FMAP_CUDA(cudaMemset(B->d_err, 0, sizeof(uint32_t)));
    set_error("in an instance: " + dev_err_message(bits));
    return dev_err_status(bits);
  }
  return FMAP_OK;
}

fmap_status fmap_batch_info(fmap_batch_t* B, int32_t* n_waves, int64_t* launches_per_run,
                            size_t* workspace_bytes, int32_t* occupancy /*[14] nullable*/,
                            int32_t* rec_templates_per_block) {
  if (!B) return batch_fail("batch is NULL");
  if (n_waves) *n_waves = (int32_t)B->waves.size();
  if (launches_per_run) *launches_per_run = B->n_launches;
  if (workspace_bytes) *workspace_bytes = B->ws_bytes;
  if (occupancy)
    for (int ph = 0; ph < BP_COUNT; ++ph) occupancy[ph] = B->tune.occ[ph];
  if (rec_templates_per_block) *rec_templates_per_block = B->tune.rec_tpb;
  return FMAP_OK;
}

fmap_status fmap_batch_profile(fmap_batch_t* B, fmap_stream stream, float* phase_ms) {
  set_error("");
  if (!B || !phase_ms) return batch_fail("fmap_batch_profile: NULL argument");
  static_assert(FMAP_BATCH_N_PHASES == BP_COUNT, "phase count");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t launches = B->n_launches;
  std::vector<cudaEvent_t> ev(2 * B->waves.size() * BP_COUNT, nullptr);
  for (auto& e : ev) FMAP_CUDA(cudaEventCreate(&e));
  fmap_status st = FMAP_OK;
  for (size_t w = 0; w < B->waves.size() && st == FMAP_OK; ++w)
    for (int ph = 0; ph < BP_COUNT && st == FMAP_OK; ++ph) {
      cudaEventRecord(ev[2 * (w * BP_COUNT + ph)], s);
      st = enqueue_phase(B, (int)w, ph, B->tune.occ[ph], s);
      cudaEventRecord(ev[2 * (w * BP_COUNT + ph) + 1], s);
    }
  cudaError_t e = cudaStreamSynchronize(s);
  if (st == FMAP_OK && e != cudaSuccess) st = cuda_fail(e, "fmap_batch_profile");
  for (size_t w = 0; w < B->waves.size() && st == FMAP_OK; ++w)
    for (int ph = 0; ph < BP_COUNT; ++ph) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * (w * BP_COUNT + ph)], ev[2 * (w * BP_COUNT + ph) + 1]);
      phase_ms[ph] += ms;
    }
  for (auto& x : ev) cudaEventDestroy(x);
  B->n_launches = launches;
  return st;
}

void fmap_batch_destroy(fmap_batch_t* B) {
  if (!B) return;
  cudaStreamSynchronize(B->cap);
  batch_free(B);
}

}  // extern "C"
