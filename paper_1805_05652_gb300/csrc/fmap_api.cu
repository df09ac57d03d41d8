// Host side of libfmap: plans, validation, workspace layout, dispatch of the
// compute paths and the C ABI of include/fmap.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fmap_internal.h"

namespace fmap {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

std::string dev_err_message(uint32_t bits) {
  std::string m;
  if (bits & DEV_ERR_ORDER) m += "timestamps are not strictly increasing; ";
  if (bits & DEV_ERR_SPAN) m += "timestamp span is >= 2^31 s; ";
  if (bits & DEV_ERR_TIMEOUT) m += "a bounded device wait gave up; ";
  if (bits & DEV_ERR_NONFINITE) m += "an atom is NaN or infinite; ";
  return m;
}

fmap_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return FMAP_ERR_CUDA;
}

static fmap_status arg_fail(const std::string& msg) {
  set_error(msg);
  return FMAP_ERR_ARG;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Grid checks (Eq. Fmn with integer seconds).
static bool grid_valid(const fmap_grid* g, std::string* why) {
  if (!g) return *why = "grid is NULL", false;
  if (g->n_t0 < 0 || g->n_tau < 0) return *why = "n_t0 and n_tau must be >= 0", false;
  if (g->window != FMAP_RECT && g->window != FMAP_EXP && g->window != FMAP_TABLE)
    return *why = "unknown window", false;
  if (g->t_sft <= 0) return *why = "t_sft must be > 0", false;
  if (g->tau_min <= 0) return *why = "tau_min must be > 0", false;
  if (g->n_tau > 1 && g->dtau <= 0) return *why = "dtau must be > 0 when n_tau > 1", false;
  if (g->n_t0 > 1 && g->dt0 <= 0) return *why = "dt0 must be > 0 when n_t0 > 1", false;
  const int64_t cells = (int64_t)g->n_t0 * g->n_tau;
  if (cells >= (int64_t)0x7fffffff) return *why = "n_t0 * n_tau must be < 2^31", false;
  const double tau_max = (double)g->tau_min + (double)std::max(0, g->n_tau - 1) * (double)g->dtau;
  if (g->window != FMAP_RECT && (g->exp_cut8 < 0 || g->exp_cut8 > 1024))
    return *why = "exp_cut8 must be in 0..1024", false;
  const double lmax = g->window == FMAP_RECT ? tau_max : tau_max * exp_cut8_of(*g) / 8.0;
  if (lmax >= 2147483647.0) return *why = "the window length at tau_max must be < 2^31 s", false;
  const double t0_ext = std::fabs((double)g->t0_min) +
                        (double)std::max(0, g->n_t0 - 1) * std::fabs((double)g->dt0);
  if (t0_ext > 4.0e18) return *why = "t0 grid out of int64 range", false;
  return true;
}

bool grid_is_valid(const fmap_grid* g, std::string* why) { return grid_valid(g, why); }

// Terms (atoms summed over the windows with >= 2 atoms) and such cells of a
// grid, uniform or with explicit axes ax (t0 values, then tau values); host.
static void count_terms_of(const fmap_grid& g, const int64_t* ax, const int64_t* t, int32_t n_sft,
                           int64_t* n_terms, int64_t* n_cells_2plus) {
  int64_t terms = 0, cells2 = 0;
  for (int32_t m = 0; m < g.n_t0; ++m) {
    const int64_t t0 = ax ? ax[m] : g.t0_min + (int64_t)m * g.dt0;
    const int64_t i0 = std::lower_bound(t, t + n_sft, t0) - t;
    int64_t j = i0;
    for (int32_t nn = 0; nn < g.n_tau; ++nn) {
      const int64_t tau = ax ? ax[g.n_t0 + nn] : g.tau_min + (int64_t)nn * g.dtau;
      const int64_t lim = t0 + window_len(g, tau) - g.t_sft;
      while (j < n_sft && t[j] <= lim) ++j;
      const int64_t c = j - i0;
      if (c >= 2) {
        terms += c;
        ++cells2;
      }
    }
  }
  *n_terms = terms;
  *n_cells_2plus = cells2;
}

static bool precision_supported(int window, fmap_precision prec) {
  if (window == FMAP_RECT) return prec == FMAP_FP64 || prec == FMAP_FP32;
  if (prec == FMAP_TF32 || prec == FMAP_BF16X3) return exp_tc_available(prec);
  return prec == FMAP_FP64 || prec == FMAP_FP32;
}

struct Layout {
  size_t rel_t, t_base, dev_err, i0, jend, coef, parts, groups, flag_blocks, n_flag, flag_list, pa, px,
      esuf, xop, perm_ant, perm_x, perm_gap, rec_cells, rec_decay, tauc, ax, wtab, flag_bits, tstat, ref_hist, ref_bin,
      ref_n, ref_cell, ref_fast, ref_val, own_map, ref_ntile, ref_tile, ref_ncand, ref_cand, total;
  int64_t n_tiles;
  int32_t tau_chunk;
};

static constexpr size_t kEsufBudget = size_t(1) << 30;

static Layout layout_of(const fmap_grid* g, int32_t n_sft, int32_t T, fmap_precision prec,
                        uint32_t flags) {
  Layout L{};
  const size_t A = 256;
  const int64_t cells = (int64_t)g->n_t0 * g->n_tau;
  const int64_t t_ant = (flags & FMAP_PLAN_PER_TEMPLATE_ANTENNA) ? T : 1;
  int64_t tiles = std::max<int64_t>(marg_tiles(*g), 1);
  if (g->window == FMAP_RECT) {
    tiles = std::max<int64_t>(tiles, rect_tiles(*g));
    tiles = std::max<int64_t>(tiles, (g->n_t0 + 127) / 128);
  } else {
    tiles = std::max<int64_t>(tiles, exp_tiles(*g));
    if (flags & FMAP_PLAN_EXP_RECURRENCE) tiles = std::max<int64_t>(tiles, g->n_tau);
  }
  L.n_tiles = tiles;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + std::max<size_t>(bytes, 1), A);
    return at;
  };
  L.rel_t = take(sizeof(int32_t) * (size_t)rel_t_entries(n_sft));
  L.t_base = take(sizeof(int64_t));
  L.dev_err = take(sizeof(uint32_t));
  L.i0 = take(sizeof(int32_t) * std::max<int32_t>(g->n_t0, 1));
  L.jend = take(sizeof(int32_t) * std::max<int64_t>(cells, 1));
  L.ax = take(sizeof(int64_t) * std::max<int64_t>((int64_t)g->n_t0 + g->n_tau, 1));
  L.parts = take(sizeof(Partial) * (size_t)std::max<int32_t>(T, 1) * (size_t)(tiles + kFixSlots));
  L.groups = take(kGroupBytes * (size_t)std::max<int32_t>(T, 1) *
                  (size_t)reduce_groups_of(tiles + kFixSlots));
  const size_t entries = (size_t)std::max<int64_t>(cells, 1) * (size_t)t_ant;
  L.coef = take(sizeof(Coef) * entries);
  L.flag_blocks = take(sizeof(int32_t) * ((entries + kFlagUnit - 1) / kFlagUnit));
  L.flag_bits = take(sizeof(uint32_t) * (size_t)flag_words((int64_t)entries));
  L.n_flag = take(sizeof(int32_t));
  L.flag_list = take(sizeof(int64_t) * entries);
  if (!(flags & kPlanBatch)) {  // refinement of the summaries
    const size_t Tn = (size_t)std::max<int32_t>(T, 1);
    L.tstat = take(sizeof(TStat) * Tn);
    L.ref_hist = take(sizeof(int32_t) * kRefBins * Tn);
    L.ref_ntile = take(sizeof(int32_t) * Tn);
    L.ref_tile = take(sizeof(int32_t) * kRefMaxTiles * Tn);
    L.ref_bin = take(sizeof(int32_t) * Tn);
    L.ref_n = take(sizeof(int32_t) * Tn);
    L.ref_ncand = take(sizeof(int32_t) * Tn);
    L.ref_cand = take(sizeof(int32_t) * kRefCandCap * Tn);
    L.ref_cell = take(sizeof(int32_t) * kRefMaxCells * Tn);
    L.ref_fast = take(sizeof(float) * kRefMaxCells * Tn);
    L.ref_val = take(sizeof(double) * kRefMaxCells * Tn);
    L.own_map = (flags & FMAP_PLAN_MAP_BUFFER)
                    ? take(sizeof(float) * (size_t)std::max<int64_t>(cells, 1) * Tn) : 0;
  }
  L.pa = L.px = L.esuf = L.xop = L.perm_ant = L.perm_x = L.perm_gap = L.rec_cells =
      L.rec_decay = L.tauc = L.wtab = 0;
  const size_t np1 = (size_t)n_sft + 1;
  if (g->window == FMAP_RECT) {
    L.pa = take(sizeof(float) * 8 * np1 * (size_t)t_ant);   // (a2, b2, ab, 0) float pairs
    L.px = take(2 * sizeof(float4) * np1 * (size_t)std::max<int32_t>(T, 1));
  } else {
    const size_t per_tau = 3 * sizeof(float2) * np1;
    int64_t chunk = (int64_t)std::max<size_t>(1, kEsufBudget / per_tau);
    chunk = std::min<int64_t>(chunk, std::max<int32_t>(g->n_tau, 1));
    L.tau_chunk = (int32_t)chunk;
    // the suffix sums live in shared memory when the data set fits there
    L.esuf = take(exp_antenna_fits(n_sft) ? 8 : per_tau * (size_t)chunk);
    const size_t perm = sizeof(float4) * (size_t)perm_entries_max(n_sft);
    L.perm_ant = take(perm * (size_t)t_ant);
    if (flags & FMAP_PLAN_EXP_RECURRENCE) {
      L.perm_x = take(perm * (size_t)std::max<int32_t>(T, 1));
      L.perm_gap = take(sizeof(int32_t) * (size_t)perm_entries_max(n_sft));
      // window records (and the shared antenna's coefficients) re-read by
      // every template after the first
      if (T >= 2 && !(flags & kPlanBatch)) {
        L.rec_cells = take((t_ant == 1 ? 2 : 1) * sizeof(float4) * (size_t)std::max<int64_t>(cells, 1));
        L.rec_decay = take(sizeof(float) * (size_t)perm_entries_max(n_sft) *
                           (size_t)std::max<int32_t>(g->n_tau, 1));
      }
    }
    L.tauc = take(sizeof(TauTab) * (size_t)std::max<int32_t>(g->n_tau, 1));
    if (g->window == FMAP_TABLE) L.wtab = take(sizeof(float2) * (kTabMax + 1));
    if (prec == FMAP_TF32 || prec == FMAP_BF16X3)
      L.xop = take(exp_tc_operand_bytes(*g, n_sft, T, prec));
  }
  L.total = off;
  return L;
}

}  // namespace fmap

using namespace fmap;

static_assert(sizeof(fmap_summary) == 32, "fmap_summary layout");
static_assert(sizeof(fmap_grid) == 64, "fmap_grid layout");
static_assert(sizeof(fmap_atoms) == 40, "fmap_atoms layout");

extern "C" {

const char* fmap_status_string(fmap_status s) {
  switch (s) {
    case FMAP_OK: return "FMAP_OK";
    case FMAP_PENDING: return "FMAP_PENDING";
    case FMAP_ERR_ARG: return "FMAP_ERR_ARG";
    case FMAP_ERR_NOMEM: return "FMAP_ERR_NOMEM";
    case FMAP_ERR_CUDA: return "FMAP_ERR_CUDA";
    case FMAP_ERR_TIMEOUT: return "FMAP_ERR_TIMEOUT";
    case FMAP_ERR_BUSY: return "FMAP_ERR_BUSY";
    case FMAP_ERR_DATA: return "FMAP_ERR_DATA";
    case FMAP_ERR_UNSUPPORTED: return "FMAP_ERR_UNSUPPORTED";
    case FMAP_ERR_NONFINITE: return "FMAP_ERR_NONFINITE";
  }
  return "FMAP_UNKNOWN";
}

const char* fmap_last_error(void) { return g_last_error.c_str(); }

size_t fmap_workspace_bytes(const fmap_grid* grid, int32_t n_sft, int32_t n_templates,
                            fmap_precision precision) {
  std::string why;
  if (!grid_valid(grid, &why) || n_sft < 0 || n_templates < 0) return 0;
  return layout_of(grid, n_sft, n_templates, precision, 0).total;
}

}  // extern "C"

namespace fmap {

// Validation shared by every way of making a plan.
static fmap_status plan_args_ok(const fmap_grid* grid, int32_t n_sft, int32_t n_templates,
                                fmap_precision precision, uint32_t flags) {
  std::string why;
  if (!grid_valid(grid, &why)) return arg_fail(why);
  if (n_sft < 0) return arg_fail("n_sft must be >= 0");
  if (n_templates < 0 || n_templates > 65535) return arg_fail("n_templates must be in [0, 65535]");
  if (precision < FMAP_FP64 || precision > FMAP_BF16X3) return arg_fail("unknown precision");
  if (flags & ~(uint32_t)(FMAP_PLAN_PER_TEMPLATE_ANTENNA | FMAP_PLAN_EXP_RECURRENCE |
                          FMAP_PLAN_MAP_BUFFER | FMAP_PLAN_GRAPH | kPlanBatch))
    return arg_fail("unknown plan flags");
  if (flags & FMAP_PLAN_EXP_RECURRENCE) {
    if (grid->window != FMAP_EXP) return arg_fail("FMAP_PLAN_EXP_RECURRENCE is for exponential windows");
    if (precision != FMAP_FP64)
      return arg_fail("FMAP_PLAN_EXP_RECURRENCE computes in compensated FP32 (FMAP_FP64 class)");
    if (!exp_rec_supported(n_sft, grid->n_t0)) {
      set_error("FMAP_PLAN_EXP_RECURRENCE keeps a template's suffix sums in shared memory: "
                "n_sft > 9000");
      return FMAP_ERR_UNSUPPORTED;
    }
  }
  if (!precision_supported(grid->window, precision)) {
    set_error("precision not offered for this window (tensor-core forms are exp-only)");
    return FMAP_ERR_UNSUPPORTED;
  }
  return FMAP_OK;
}

fmap_status plan_footprint(const fmap_grid* grid, int32_t n_sft, int32_t n_templates,
                           fmap_precision precision, uint32_t flags, size_t* bytes) {
  const fmap_status st = plan_args_ok(grid, n_sft, n_templates, precision, flags);
  if (st != FMAP_OK) return st;
  *bytes = layout_of(grid, n_sft, n_templates, precision, flags).total;
  return FMAP_OK;
}

fmap_status plan_init(fmap_plan_s* p, const fmap_grid* grid, int32_t n_sft, int32_t n_templates,
                      fmap_precision precision, uint32_t flags, void* base, size_t bytes) {
  fmap_status st = plan_args_ok(grid, n_sft, n_templates, precision, flags);
  if (st != FMAP_OK) return st;
  p->grid = *grid;
  p->n_sft = n_sft;
  p->n_templates = n_templates;
  p->precision = precision;
  p->flags = flags;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  const Layout L = layout_of(grid, n_sft, n_templates, precision, flags);
  if (!base || bytes < L.total) return arg_fail("workspace smaller than the plan's footprint");
  p->n_tiles = L.n_tiles;
  p->part_stride = L.n_tiles + kFixSlots;
  p->tau_chunk = L.tau_chunk;
  char* b = (char*)base;
  Workspace& w = p->ws;
  w.base = base;
  w.bytes = L.total;
  w.rel_t = (int32_t*)(b + L.rel_t);
  w.t_base = (int64_t*)(b + L.t_base);
  w.dev_err = (uint32_t*)(b + L.dev_err);
  w.i0 = (int32_t*)(b + L.i0);
  w.jend = (int32_t*)(b + L.jend);
  w.ax = (int64_t*)(b + L.ax);
  w.partials = (Partial*)(b + L.parts);
  w.groups = (void*)(b + L.groups);
  w.coef = (Coef*)(b + L.coef);
  w.flag_blocks = (int32_t*)(b + L.flag_blocks);
  w.flag_bits = (uint32_t*)(b + L.flag_bits);
  w.n_flag = (int32_t*)(b + L.n_flag);
  w.flag_list = (int64_t*)(b + L.flag_list);
  if (!(flags & kPlanBatch)) {
    w.tstat = (TStat*)(b + L.tstat);
    w.ref_hist = (int32_t*)(b + L.ref_hist);
    w.ref_ntile = (int32_t*)(b + L.ref_ntile);
    w.ref_tile = (int32_t*)(b + L.ref_tile);
    w.ref_bin = (int32_t*)(b + L.ref_bin);
    w.ref_n = (int32_t*)(b + L.ref_n);
    w.ref_ncand = (int32_t*)(b + L.ref_ncand);
    w.ref_cand = (int32_t*)(b + L.ref_cand);
    w.ref_cell = (int32_t*)(b + L.ref_cell);
    w.ref_fast = (float*)(b + L.ref_fast);
    w.ref_val = (double*)(b + L.ref_val);
    w.own_map = (flags & FMAP_PLAN_MAP_BUFFER) ? (float*)(b + L.own_map) : nullptr;
  } else {
    p->refine_cells = 0;
  }
  if (grid->window == FMAP_RECT) {
    w.pa = (float4*)(b + L.pa);
    w.px = (float4*)(b + L.px);
  } else {
    w.esuf = (float2*)(b + L.esuf);
    w.perm_ant = (float4*)(b + L.perm_ant);
    if (L.perm_x) w.perm_x = (float4*)(b + L.perm_x);
    if (L.perm_gap) w.perm_gap = (int32_t*)(b + L.perm_gap);
    if (L.rec_cells) w.rec_cells = (float4*)(b + L.rec_cells);
    if (L.rec_decay) w.rec_decay = (float*)(b + L.rec_decay);
    if (L.wtab) w.wtab = (float2*)(b + L.wtab);
    w.tauc = (TauTab*)(b + L.tauc);
    if (L.xop) w.xop = (void*)(b + L.xop);
  }
  p->needs_err_reset = true;
  return FMAP_OK;
}

}  // namespace fmap

extern "C" {

fmap_status fmap_plan(fmap_plan_t** out, const fmap_grid* grid, int32_t n_sft,
                      int32_t n_templates, fmap_precision precision, uint32_t flags) {
  set_error("");
  if (!out) return arg_fail("plan output pointer is NULL");
  *out = nullptr;
  if (flags & kPlanBatch) return arg_fail("unknown plan flags");   // (internal to batches)
  size_t total = 0;
  fmap_status st = plan_footprint(grid, n_sft, n_templates, precision, flags, &total);
  if (st != FMAP_OK) return st;
  fmap_plan_s* p = new (std::nothrow) fmap_plan_s();
  if (!p) return FMAP_ERR_NOMEM;
  void* base = nullptr;
  cudaError_t e = cudaMalloc(&base, total);
  if (e != cudaSuccess) {
    delete p;
    cudaGetLastError();
    set_error("workspace allocation of " + std::to_string(total) + " bytes failed");
    return FMAP_ERR_NOMEM;
  }
  st = plan_init(p, grid, n_sft, n_templates, precision, flags, base, total);
  if (st != FMAP_OK) {
    cudaFree(base);
    delete p;
    return st;
  }
  p->owns_ws = true;
  *out = p;
  return FMAP_OK;
}

static void drop_events(fmap_plan_s* p) {
  for (auto e : p->events) cudaEventDestroy(e);
  p->events.clear();
}

static void free_staging(fmap_plan_s* p) {
  Workspace& w = p->ws;
  cudaFree(w.st_t);
  cudaFree(w.st_ant);
  cudaFree(w.st_x);
  cudaFree(w.st_map);
  cudaFree(w.st_sum);
  w.st_t = nullptr;
  w.st_ant = w.st_x = w.st_map = nullptr;
  w.st_sum = nullptr;
}

}  // extern "C"

namespace fmap {
void plan_release(fmap_plan_s* p) {
  drop_events(p);
  free_staging(p);
  if (p->graph) cudaGraphExecDestroy(p->graph);
  p->graph = nullptr;
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  p->cap_stream = nullptr;
}
}  // namespace fmap

extern "C" {

void fmap_plan_destroy(fmap_plan_t* p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != p->device) cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  plan_release(p);
  if (p->owns_ws) cudaFree(p->ws.base);
  if (cur != p->device) cudaSetDevice(cur);
  delete p;
}

fmap_status fmap_plan_set_log_prior(fmap_plan_t* p, double c) {
  if (!p) return arg_fail("plan is NULL");
  if (!std::isfinite(c)) return arg_fail("log prior constant must be finite");
  p->log_prior = c;
  p->graph_key_window = -1;   // (a captured graph holds the old value)
  return FMAP_OK;
}

static fmap_status check_atoms(const fmap_plan_s* p, const fmap_atoms* a) {
  if (!a) return arg_fail("atoms is NULL");
  if (a->n_sft != p->n_sft) return arg_fail("atoms.n_sft differs from the plan");
  if (a->n_templates != p->n_templates) return arg_fail("atoms.n_templates differs from the plan");
  if (!a->shared_antenna && !(p->flags & FMAP_PLAN_PER_TEMPLATE_ANTENNA))
    return arg_fail("per-template antenna rows need a plan made with FMAP_PLAN_PER_TEMPLATE_ANTENNA");
  if (p->n_sft > 0 && (!a->t || !a->antenna || (p->n_templates > 0 && !a->fafb)))
    return arg_fail("atom pointers must be non-NULL when n_sft > 0");
  return FMAP_OK;
}

static fmap_status check_device(const fmap_plan_s* p) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != p->device) return arg_fail("current device differs from the plan's device");
  return FMAP_OK;
}

static fmap_status enqueue(fmap_plan_t* p, const fmap_atoms* a, float* d_2F,
                           fmap_summary* d_summary, cudaStream_t s, int window,
                           const cudaEvent_t* evp);

static fmap_status compute(fmap_plan_t* p, const fmap_atoms* a, float* d_2F,
                           fmap_summary* d_summary, cudaStream_t s, int window) {
  set_error("");
  if (!p) return arg_fail("plan is NULL");
  if (p->grid.window != window)
    return arg_fail("the plan's grid window does not match this compute call");
  if (window == FMAP_TABLE && p->n_tab < 2)
    return arg_fail("fmap_plan_window_table has not been called on this plan");
  fmap_status st = check_atoms(p, a);
  if (st != FMAP_OK) return st;
  st = check_device(p);
  if (st != FMAP_OK) return st;
  p->last_stream = s;
  if (!d_2F && !d_summary) return FMAP_OK;
  // summary-only calls write the plan's own map when it has one, so that the
  // summaries can be refined
  if (!d_2F && p->ws.own_map) d_2F = p->ws.own_map;
  if (p->needs_err_reset) {   // (outside any graph: an unread error is kept)
    FMAP_CUDA(cudaMemsetAsync(p->ws.dev_err, 0, sizeof(uint32_t), s));
    p->needs_err_reset = false;
  }
  if ((p->flags & FMAP_PLAN_GRAPH) && !p->timing) {
    const void* key[6] = {a->t, a->antenna, a->fafb, (const void*)(intptr_t)a->shared_antenna,
                          d_2F, d_summary};
    bool same = p->graph && p->graph_key_window == window;
    for (int k = 0; k < 6 && same; ++k) same = key[k] == p->graph_key[k];
    if (!same) {
      if (p->graph) {   // (the old graph may still be running)
        FMAP_CUDA(cudaStreamSynchronize(p->graph_stream));
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
      }
      if (!p->cap_stream) FMAP_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
      FMAP_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
      const int64_t l0 = p->launches;
      const fmap_status st_e = enqueue(p, a, d_2F, d_summary, p->cap_stream, window, nullptr);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
      if (st_e != FMAP_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st_e != FMAP_OK ? st_e : cuda_fail(e, "cudaStreamEndCapture");
      }
      const cudaError_t ei = cudaGraphInstantiate(&p->graph, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) {
        p->graph = nullptr;
        return cuda_fail(ei, "cudaGraphInstantiate");
      }
      for (int k = 0; k < 6; ++k) p->graph_key[k] = key[k];
      p->graph_key_window = window;
      p->graph_launches = p->launches - l0;
      p->launches = l0;
    }
    FMAP_CUDA(cudaGraphLaunch(p->graph, s));
    p->graph_stream = s;
    p->launches += p->graph_launches;
    return FMAP_OK;
  }
  cudaEvent_t ev[FMAP_N_PHASES + 1] = {};
  if (p->timing) {
    for (auto& e : ev) FMAP_CUDA(cudaEventCreate(&e));
    for (auto e : ev) p->events.push_back(e);
    FMAP_CUDA(cudaEventRecord(ev[0], s));
  }
  return enqueue(p, a, d_2F, d_summary, s, window, ev);
}

// The launches of one compute call on stream s (ev: the phase events of a
// timed call, else null).
static fmap_status enqueue(fmap_plan_t* p, const fmap_atoms* a, float* d_2F,
                           fmap_summary* d_summary, cudaStream_t s, int window,
                           const cudaEvent_t* evp) {
  cudaEvent_t ev[FMAP_N_PHASES + 1] = {};
  if (evp)
    for (int k = 0; k <= FMAP_N_PHASES; ++k) ev[k] = evp[k];
  FMAP_CUDA(launch_prep(p, a, s));
  {   // the bitmask of ill-conditioned entries, set by the coefficient kernels
    const int64_t ent = (int64_t)p->grid.n_t0 * p->grid.n_tau *
                        (a->shared_antenna ? 1 : std::max<int32_t>(p->n_templates, 1));
    if (ent > 0)
      FMAP_CUDA(cudaMemsetAsync(p->ws.flag_bits, 0, sizeof(uint32_t) * (size_t)flag_words(ent), s));
  }
  FMAP_CUDA(launch_index(p, a->t, s));
  if (ev[1]) FMAP_CUDA(cudaEventRecord(ev[1], s));
  int64_t tiles = 0;
  if (window == FMAP_RECT) {
    FMAP_CUDA(launch_rect_coef(p, a, s));
    FMAP_CUDA(launch_rect(p, a, d_2F, s, &tiles, ev[2]));
  } else if (window == FMAP_TABLE) {
    FMAP_CUDA(launch_table_antenna(p, a, s));
    if (ev[2]) FMAP_CUDA(cudaEventRecord(ev[2], s));
    if (p->precision == FMAP_TF32 || p->precision == FMAP_BF16X3)
      FMAP_CUDA(launch_exp_tc(p, a, d_2F, s, &tiles));
    else
      FMAP_CUDA(launch_exp_plain(p, a, d_2F, s, &tiles));
  } else {
    FMAP_CUDA(launch_exp_perm(p, a, s));
    FMAP_CUDA(launch_exp_coef(p, a, s));
    if (ev[2]) FMAP_CUDA(cudaEventRecord(ev[2], s));
    if (p->flags & FMAP_PLAN_EXP_RECURRENCE) {
      FMAP_CUDA(launch_exp_rec(p, a, d_2F, s, &tiles));
    } else if (p->precision == FMAP_TF32 || p->precision == FMAP_BF16X3) {
      FMAP_CUDA(launch_exp_tc(p, a, d_2F, s, &tiles));
    } else {
      FMAP_CUDA(launch_exp_plain(p, a, d_2F, s, &tiles));
    }
  }
  if (ev[3]) FMAP_CUDA(cudaEventRecord(ev[3], s));
  FMAP_CUDA(launch_flag_and_fixup(p, a, d_2F, s));
  FMAP_CUDA(launch_final_reduce(p, tiles, true, d_summary, s));
  FMAP_CUDA(launch_refine(p, a, d_2F, d_summary, tiles, s));
  if (ev[4]) FMAP_CUDA(cudaEventRecord(ev[4], s));
  return FMAP_OK;
}

fmap_status fmap_compute_rect(fmap_plan_t* p, const fmap_atoms* a, float* d_2F,
                              fmap_summary* d_summary, fmap_stream stream) {
  return compute(p, a, d_2F, d_summary, (cudaStream_t)stream, FMAP_RECT);
}

fmap_status fmap_compute_exp(fmap_plan_t* p, const fmap_atoms* a, float* d_2F,
                             fmap_summary* d_summary, fmap_stream stream) {
  return compute(p, a, d_2F, d_summary, (cudaStream_t)stream, FMAP_EXP);
}

fmap_status fmap_compute_table(fmap_plan_t* p, const fmap_atoms* a, float* d_2F,
                               fmap_summary* d_summary, fmap_stream stream) {
  return compute(p, a, d_2F, d_summary, (cudaStream_t)stream, FMAP_TABLE);
}

fmap_status fmap_plan_window_table(fmap_plan_t* p, const float* w, int32_t n_points) {
  set_error("");
  if (!p) return arg_fail("plan is NULL");
  if (p->grid.window != FMAP_TABLE) return arg_fail("the plan's grid is not an FMAP_TABLE grid");
  if (!w || n_points < 2 || n_points > kTabMax) return arg_fail("need 2..1024 window samples");
  for (int32_t k = 0; k < n_points; ++k)
    if (!std::isfinite(w[k])) return arg_fail("window samples must be finite");
  if (p->last_stream) FMAP_CUDA(cudaStreamSynchronize(p->last_stream));
  // (w_k, w_{k+1} - w_k) per sample interval, (w_last, 0), then the zero sentinel
  std::vector<float2> tab((size_t)n_points + 1);
  for (int32_t k = 0; k < n_points; ++k)
    tab[k] = make_float2(w[k], k + 1 < n_points ? w[k + 1] - w[k] : 0.0f);
  tab[n_points] = make_float2(0.0f, 0.0f);
  FMAP_CUDA(cudaMemcpy(p->ws.wtab, tab.data(), sizeof(float2) * tab.size(), cudaMemcpyHostToDevice));
  p->n_tab = n_points;
  p->graph_key_window = -1;   // (a captured graph holds the old table size)
  return FMAP_OK;
}

fmap_status fmap_marginalise(fmap_plan_t* p, const float* d_2F, const uint8_t* d_valid,
                             fmap_summary* d_summary, fmap_stream stream) {
  set_error("");
  if (!p) return arg_fail("plan is NULL");
  const int64_t cells = (int64_t)p->grid.n_t0 * p->grid.n_tau;
  if (!d_summary) return arg_fail("summary output is NULL");
  if (cells > 0 && p->n_templates > 0 && !d_2F) return arg_fail("map is NULL");
  fmap_status st = check_device(p);
  if (st != FMAP_OK) return st;
  p->last_stream = (cudaStream_t)stream;
  if (p->needs_err_reset) {
    FMAP_CUDA(cudaMemsetAsync(p->ws.dev_err, 0, sizeof(uint32_t), (cudaStream_t)stream));
    p->needs_err_reset = false;
  }
  FMAP_CUDA(launch_marginalise(p, d_2F, d_valid, d_summary, (cudaStream_t)stream));
  return FMAP_OK;
}

fmap_status fmap_plan_enable_timing(fmap_plan_t* p, int32_t enable) {
  if (!p) return arg_fail("plan is NULL");
  drop_events(p);
  p->timing = enable != 0;
  p->launches = 0;
  return FMAP_OK;
}

fmap_status fmap_plan_read_timing(fmap_plan_t* p, double* ms, int64_t* calls, int64_t* launches) {
  if (!p) return arg_fail("plan is NULL");
  const size_t per = FMAP_N_PHASES + 1;
  double acc[FMAP_N_PHASES] = {0, 0, 0, 0};
  const size_t n_calls = p->events.size() / per;
  for (size_t c = 0; c < n_calls; ++c) {
    cudaEvent_t* e = &p->events[c * per];
    FMAP_CUDA(cudaEventSynchronize(e[per - 1]));
    for (int k = 0; k < FMAP_N_PHASES; ++k) {
      float t = 0.f;
      FMAP_CUDA(cudaEventElapsedTime(&t, e[k], e[k + 1]));
      acc[k] += t;
    }
  }
  if (ms)
    for (int k = 0; k < FMAP_N_PHASES; ++k) ms[k] = acc[k];
  if (calls) *calls = (int64_t)n_calls;
  if (launches) *launches = p->launches;
  return FMAP_OK;
}

fmap_status fmap_plan_status(fmap_plan_t* p) {
  if (!p) return arg_fail("plan is NULL");
  FMAP_CUDA(cudaStreamSynchronize(p->last_stream));
  uint32_t bits = 0;
  FMAP_CUDA(cudaMemcpy(&bits, p->ws.dev_err, sizeof(bits), cudaMemcpyDeviceToHost));
  if (bits) {
    FMAP_CUDA(cudaMemset(p->ws.dev_err, 0, sizeof(uint32_t)));
    set_error(dev_err_message(bits));
    return dev_err_status(bits);
  }
  return FMAP_OK;
}

fmap_status fmap_plan_set_refine(fmap_plan_t* p, int32_t max_cells) {
  set_error("");
  if (!p) return arg_fail("plan is NULL");
  if (max_cells > kRefMaxCells) return arg_fail("at most 4096 refined cells per template");
  p->refine_cells = max_cells < 0 ? -1 : max_cells;
  p->graph_key_window = -1;   // (a captured graph holds the old value)
  return FMAP_OK;
}

fmap_status fmap_plan_set_wait_limit(fmap_plan_t* p, int64_t limit_ns) {
  set_error("");
  if (!p) return arg_fail("plan is NULL");
  p->wait_ns = limit_ns < 0 ? kDefaultWaitNs : limit_ns;
  p->graph_key_window = -1;   // (a captured graph holds the old value)
  return FMAP_OK;
}

fmap_status fmap_combine_summaries(const fmap_summary* shards, int32_t n_shards,
                                   int32_t n_templates, const int32_t* m_offsets,
                                   fmap_summary* out) {
  set_error("");
  if (n_shards < 0 || n_templates < 0) return arg_fail("negative shard or template count");
  if (n_templates > 0 && (!out || (n_shards > 0 && (!shards || !m_offsets))))
    return arg_fail("NULL shards, offsets or output");
  for (int32_t j = 0; j < n_templates; ++j) {
    int64_t n_tot = 0;
    bool have = false;
    float best = 0.0f;
    int64_t bm = -1, bn = -1;
    int32_t flags = ~0;
    double hi = -INFINITY;
    std::vector<double> terms;
    terms.reserve((size_t)n_shards);
    for (int32_t r = 0; r < n_shards; ++r) {
      const fmap_summary& q = shards[(int64_t)r * n_templates + j];
      if (q.n_valid <= 0) continue;
      n_tot += q.n_valid;
      const int64_t gm = (int64_t)q.m + m_offsets[r], gn = q.n;
      if (!have || q.max2F > best || (q.max2F == best && (gm < bm || (gm == bm && gn < bn)))) {
        best = q.max2F;
        bm = gm;
        bn = gn;
      }
      have = true;
      flags &= q.flags;
      const double v = q.logB + std::log((double)q.n_valid);
      terms.push_back(v);
      hi = std::max(hi, v);
    }
    fmap_summary o;
    o.n_valid = n_tot;
    if (!have) {
      o.max2F = 0.0f;
      o.m = o.n = -1;
      o.flags = 0;
      o.logB = std::nan("");
    } else {
      double acc = 0.0;
      for (double v : terms) acc += std::exp(v - hi);
      o.max2F = best;
      o.m = (int32_t)bm;
      o.n = (int32_t)bn;
      o.flags = flags;
      o.logB = hi + std::log(acc) - std::log((double)n_tot);
    }
    out[j] = o;
  }
  return FMAP_OK;
}

fmap_status fmap_compute_host(fmap_plan_t* p, const fmap_atoms* h, float* h_2F,
                              fmap_summary* h_summary, fmap_stream stream) {
  set_error("");
  if (!p) return arg_fail("plan is NULL");
  fmap_status st = check_atoms(p, h);
  if (st != FMAP_OK) return st;
  st = check_device(p);
  if (st != FMAP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace& w = p->ws;
  const size_t n = (size_t)p->n_sft, T = (size_t)p->n_templates;
  const size_t n_ant = h->shared_antenna ? 1 : T;
  const size_t cells = (size_t)p->grid.n_t0 * (size_t)p->grid.n_tau;
  if (!w.st_t) {
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&w.st_t, sizeof(int64_t) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(&w.st_ant, sizeof(float) * 3 * std::max<size_t>(n, 1) *
                                                        (p->flags & FMAP_PLAN_PER_TEMPLATE_ANTENNA ? std::max<size_t>(T, 1) : 1));
    if (e == cudaSuccess) e = cudaMalloc(&w.st_x, sizeof(float) * 4 * std::max<size_t>(n * T, 1));
    if (e == cudaSuccess) e = cudaMalloc(&w.st_sum, sizeof(fmap_summary) * std::max<size_t>(T, 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_staging(p);
      set_error("staging allocation failed");
      return FMAP_ERR_NOMEM;
    }
  }
  // the map staging only when a map is asked for
  if (h_2F && !w.st_map) {
    if (cudaMalloc(&w.st_map, sizeof(float) * std::max<size_t>(cells * T, 1)) != cudaSuccess) {
      cudaGetLastError();
      w.st_map = nullptr;
      set_error("staging allocation failed");
      return FMAP_ERR_NOMEM;
    }
  }
  if (n > 0) {
    FMAP_CUDA(cudaMemcpyAsync(w.st_t, h->t, sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
    FMAP_CUDA(cudaMemcpyAsync(w.st_ant, h->antenna, sizeof(float) * 3 * n * n_ant,
                              cudaMemcpyHostToDevice, s));
    if (T > 0)
      FMAP_CUDA(cudaMemcpyAsync(w.st_x, h->fafb, sizeof(float) * 4 * n * T,
                                cudaMemcpyHostToDevice, s));
  }
  fmap_atoms d = *h;
  d.t = w.st_t;
  d.antenna = w.st_ant;
  d.fafb = w.st_x;
  st = compute(p, &d, h_2F ? w.st_map : nullptr, h_summary ? w.st_sum : nullptr, s,
               p->grid.window);
  if (st != FMAP_OK) return st;
  if (h_2F && cells * T > 0)
    FMAP_CUDA(cudaMemcpyAsync(h_2F, w.st_map, sizeof(float) * cells * T, cudaMemcpyDeviceToHost, s));
  if (h_summary && T > 0)
    FMAP_CUDA(cudaMemcpyAsync(h_summary, w.st_sum, sizeof(fmap_summary) * T,
                              cudaMemcpyDeviceToHost, s));
  FMAP_CUDA(cudaStreamSynchronize(s));
  return FMAP_OK;
}

fmap_status fmap_count_terms(const fmap_grid* g, const int64_t* t, int32_t n_sft, int64_t* n_terms,
                             int64_t* n_cells_2plus) {
  set_error("");
  std::string why;
  if (!grid_valid(g, &why)) return arg_fail(why);
  if (n_sft < 0 || (n_sft > 0 && !t)) return arg_fail("bad timestamps");
  if (!n_terms || !n_cells_2plus) return arg_fail("outputs are NULL");
  count_terms_of(*g, nullptr, t, n_sft, n_terms, n_cells_2plus);
  return FMAP_OK;
}

fmap_status fmap_plan_count_terms(fmap_plan_t* p, const int64_t* t, int32_t n_sft,
                                  int64_t* n_terms, int64_t* n_cells_2plus) {
  set_error("");
  if (!p) return arg_fail("plan is NULL");
  if (n_sft < 0 || (n_sft > 0 && !t)) return arg_fail("bad timestamps");
  if (!n_terms || !n_cells_2plus) return arg_fail("outputs are NULL");
  count_terms_of(p->grid, p->explicit_axes ? p->ax_host.data() : nullptr, t, n_sft, n_terms,
                 n_cells_2plus);
  return FMAP_OK;
}

fmap_status fmap_plan_axes(fmap_plan_t* p, const int64_t* t0_values, const int64_t* tau_values) {
  set_error("");
  if (!p) return arg_fail("plan is NULL");
  if (!t0_values != !tau_values) return arg_fail("give both axes or neither");
  if (p->last_stream) FMAP_CUDA(cudaStreamSynchronize(p->last_stream));
  p->graph_key_window = -1;   // (a captured graph holds the old axes argument)
  if (!t0_values) {
    p->explicit_axes = false;
    p->ax_host.clear();
    return FMAP_OK;
  }
  const fmap_grid& g = p->grid;
  for (int32_t m = 0; m < g.n_t0; ++m) {
    if (t0_values[m] > ((int64_t)1 << 62) || t0_values[m] < -((int64_t)1 << 62))
      return arg_fail("t0 value out of range");
    if (m > 0 && t0_values[m] <= t0_values[m - 1]) return arg_fail("t0 values must increase");
  }
  for (int32_t n = 0; n < g.n_tau; ++n) {
    if (tau_values[n] <= 0) return arg_fail("tau values must be > 0");
    if (n > 0 && tau_values[n] <= tau_values[n - 1]) return arg_fail("tau values must increase");
  }
  if (g.n_tau > 0 && (double)window_len(g, tau_values[g.n_tau - 1]) >= 2147483647.0)
    return arg_fail("the window length at the largest tau must be < 2^31 s");
  std::vector<int64_t> ax((size_t)g.n_t0 + g.n_tau);
  std::copy(t0_values, t0_values + g.n_t0, ax.begin());
  std::copy(tau_values, tau_values + g.n_tau, ax.begin() + g.n_t0);
  if (!ax.empty())
    FMAP_CUDA(cudaMemcpy(p->ws.ax, ax.data(), sizeof(int64_t) * ax.size(), cudaMemcpyHostToDevice));
  p->ax_host.swap(ax);
  p->explicit_axes = true;
  return FMAP_OK;
}

}  // extern "C"
