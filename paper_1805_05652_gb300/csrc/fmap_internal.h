// Internal declarations of libfmap: the plan, its workspace, the per-tile
// reduction partials and the device helpers every kernel shares.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fmap.h"

namespace fmap {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
fmap_status cuda_fail(cudaError_t e, const char* what);

#define FMAP_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return ::fmap::cuda_fail(e_, #call); \
  } while (0)

// Device-side error bits latched in the plan's status word.
enum : uint32_t { DEV_ERR_ORDER = 1u, DEV_ERR_SPAN = 2u, DEV_ERR_TIMEOUT = 4u,
                  DEV_ERR_NONFINITE = 8u };
// Status of latched device error bits (0 when none): a timeout first, then
// data errors, then non-finite atoms.
inline fmap_status dev_err_status(uint32_t bits) {
  if (bits & DEV_ERR_TIMEOUT) return FMAP_ERR_TIMEOUT;
  if (bits & (DEV_ERR_ORDER | DEV_ERR_SPAN)) return FMAP_ERR_DATA;
  if (bits & DEV_ERR_NONFINITE) return FMAP_ERR_NONFINITE;
  return FMAP_OK;
}
std::string dev_err_message(uint32_t bits);
// Default limit of a bounded device wait (ns).
constexpr int64_t kDefaultWaitNs = 2000000000ll;

// ---------------------------------------------------------------------------
// Reduction partial of one tile and one template.  sum = sum over the tile's
// valid cells of exp(F - F_max) with F = 2F/2 and F_max = max2F/2; arg is the
// lowest linear index m*n_tau+n holding max2F; nvalid = 0 marks an empty
// partial (max2F = -1, arg = INT32_MAX, sum = 0).
// ---------------------------------------------------------------------------
struct __align__(16) Partial {
  float max2F;
  int32_t arg;
  float sum;
  int32_t nvalid;
};

// Per-cell 2F coefficients.  2F = k1 |Fa|^2 + k2 |Fb - beta Fa|^2, which is
// Eq. (F_FaFb) times two with k1 = 2/A, beta = C/A, k2 = 2A/D (completing the
// square in Fa).  valid: 0 = invalid (fewer than 2 atoms; k1 = k2 = 0),
// 1 = evaluated by the fast kernels, 2 = ill-conditioned or undecided
// (A B / D > kCondThreshold, or D not clearly positive in float-float): left
// to the fix-up of fmap_fixup.cu, which decides D > 0 from float-float sums
// and then records the outcome in valid (3 = valid, 0 = invalid).
constexpr double kCondThreshold = 100.0;
// Reduction slots per template written by the fix-up kernel.
constexpr int kFixSlots = 512;
// Below this many templates the fix-up runs one thread per listed entry
// (else one per template), and spreads the list over just enough slots for
// about kFixPerSlot entries each (else over all kFixSlots).
constexpr int kFixCellModeT = 8;
constexpr int kFixPerSlot = 128;
// Entries [lo, hi) of fix-up slot b (of G) for a list of n entries and T
// templates; every slot past the used ones is empty.  The fix-up kernels
// and the refinement's scan of a slot's cells share this partition.
__host__ __device__ inline void fix_slot_range(int64_t b, int64_t n, int32_t G, int32_t T,
                                               int64_t* lo, int64_t* hi) {
  const int64_t per = T < kFixCellModeT ? kFixPerSlot : 1;
  int64_t used = (n + per - 1) / per;
  used = used < 1 ? 1 : (used > G ? G : used);
  *lo = b < used ? b * n / used : n;
  *hi = b < used ? (b + 1) * n / used : n;
}
// Internal plan flag (not part of the C ABI) of batch instances, whose
// workspaces are kept lean: the plan never refines its summaries (no
// refinement arrays), and the recurrence recomputes its window records per
// template (no record array).
constexpr uint32_t kPlanBatch = 1u << 16;
// Top-cell refinement (fmap_refine.cu): candidates per template (at most),
// histogram bins over the window of kRefWindow (2F units) below the maximum.
constexpr int kRefMaxCells = 4096;
// Cells per template the histogram pass may keep for the cut (those in a bin
// <= the tile pass's bound); a template with more is collected by a second
// scan of its tiles.
constexpr int kRefCandCap = 8192;
constexpr int kRefBins = 256;
constexpr float kRefWindow = 16.0f;
// Tiles the refinement may scan per template (those whose fast maximum can
// bound a top cell; a few more than the cells wanted, ties included).
constexpr int kRefMaxTiles = 16384;
// Geometry of the reduction tiles of a plan's main kernel: rectangles of R
// t0 rows x C tau columns, tile index tr * ntc + tc (row-major) or tc * ntr +
// tr (column-major), so that a tile's cells can be found from its index.
struct TileGeom {
  int32_t col_major;
  int32_t R, C;
  int32_t ntr, ntc;
};
// Per-template statistics of the fast reduction, kept for the refinement:
// S = sum over valid cells of exp((2F - M) / 2), M = max 2F, arg its lowest
// cell, N the valid count.
struct __align__(32) TStat {
  double S;
  float M;
  int32_t arg;
  long long N;
  long long pad;
};
// Window length L(tau) in seconds: tau (rect) or floor(cut8 tau / 8) (exp,
// cut8 = 24 by default: Eq. winexp's 3 tau).  An atom belongs to the window
// of (t0, tau) iff t0 <= t and t + T_sft <= t0 + L(tau).
__host__ __device__ inline int32_t exp_cut8_of(const fmap_grid& g) {
  return g.exp_cut8 > 0 ? g.exp_cut8 : 24;
}
__host__ __device__ inline int64_t window_len(const fmap_grid& g, int64_t tau) {
  return g.window == FMAP_RECT ? tau : (int64_t)exp_cut8_of(g) * tau / 8;
}
// Largest window table (samples) of FMAP_TABLE grids.
constexpr int kTabMax = 1024;
// Entries per count of the marked-entry compaction: one bitmask word per
// thread of a 1024-thread block.
constexpr int kFlagUnit = 32768;
// Words of the marked-entry bitmask (whole compaction units).
__host__ __device__ inline int64_t flag_words(int64_t entries) {
  return (entries + kFlagUnit - 1) / kFlagUnit * (kFlagUnit / 32);
}
// Threads of the exponential-window scans ("lanes", 64, 128 or 256, a plan
// property): thread t of a scan owns the atoms [t C, t C + C), C =
// ceil(N / lanes), and the scans read the atoms from a chunk-major copy
// (entry q lanes + t holds atom t C + q), so the loads of a warp at one chunk
// position are contiguous.  Single plans scan with 256 threads; batches, whose
// many short units favour throughput over the latency of one tau, take fewer
// for short data sets (batch_scan_lanes), so that combining the threads'
// chunks stays cheap next to the chunks themselves.
constexpr int kScanLanes = 256;   // the most threads of a scan
__host__ __device__ inline int32_t batch_scan_lanes(int32_t n_sft) {
  return n_sft <= 1024 ? 128 : 256;
}
// Atoms per thread: odd, so that the threads' chunk starts (stride C) fall
// in distinct shared-memory banks across a warp.
__host__ __device__ inline int64_t scan_chunk(int32_t n_sft, int32_t lanes) {
  return (((int64_t)n_sft + lanes - 1) / lanes) | 1;
}
__host__ __device__ inline int64_t perm_entries(int32_t n_sft, int32_t lanes) {
  return scan_chunk(n_sft, lanes) * lanes;
}
// The most entries of any scan width (workspaces take this).
__host__ __device__ inline int64_t perm_entries_max(int32_t n_sft) {
  int64_t e = perm_entries(n_sft, 64);
  e = e > perm_entries(n_sft, 128) ? e : perm_entries(n_sft, 128);
  return e > perm_entries(n_sft, 256) ? e : perm_entries(n_sft, 256);
}
// Grid values t0_m and tau_n: Eq. Fmn's uniform grid, or the plan's explicit
// axes ax (t0 values, then tau values) when given (non-null).
__host__ __device__ inline int64_t grid_t0(const fmap_grid& g, const int64_t* ax, int64_t m) {
  return ax ? ax[m] : g.t0_min + m * g.dt0;
}
__host__ __device__ inline int64_t grid_tau(const fmap_grid& g, const int64_t* ax, int64_t n) {
  return ax ? ax[g.n_t0 + n] : g.tau_min + n * g.dtau;
}
// Entries of the exp copy step: the chunk-major copies, then one per tau.
// (plan_axes, after the plan struct: the axes to pass kernels, or null.)
__host__ __device__ inline int64_t exp_copy_entries(int32_t n_sft, int32_t lanes, int32_t n_ant,
                                                    int32_t n_x, int32_t n_tau) {
  return perm_entries(n_sft, lanes) * (int64_t)(n_ant + n_x) + n_tau;
}
// Per-tau constants of the exponential window, for the weight w (s = 1) and
// the antenna weight w^2 (s = 2): the decays over gaps of k = 0..kPowTab-1
// whole SFTs as float pairs, pw[s-1][k] = e^{-s k T_sft / tau} (powers of the
// one-SFT decay in float-float), the exp2 slopes c2[s-1] = -s log2(e) / tau,
// and 1 / tau.  Filled once per plan run by the exp copy step.
constexpr int kPowTab = 16;
struct __align__(16) TauTab {
  double inv_tau;
  float c2[2];
  float2 pw[2][kPowTab];
};
struct __align__(16) Coef {
  float k1;
  float beta;
  float k2;
  float valid;
};

// Workspace of a plan (all device memory, owned by the plan).
struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
  int32_t* rel_t = nullptr;      // [round_up(N, 64) + 64] t - t[0], zero padded
  int64_t* t_base = nullptr;     // [1] t[0]
  uint32_t* dev_err = nullptr;   // [1] latched device error bits
  int32_t* i0 = nullptr;         // [n_t0] first atom with t >= t0_m
  int32_t* jend = nullptr;       // [n_t0][n_tau] one past the last atom of each window
  Coef* coef = nullptr;          // [T_ant][n_t0][n_tau]
  Partial* partials = nullptr;   // [T][n_tiles + kFixSlots]
  void* groups = nullptr;        // [T][reduce_groups_of(n_tiles + kFixSlots)] FP64 group merges
  int32_t* flag_blocks = nullptr;  // [ceil(T_ant cells / kFlagUnit)] counts, then offsets
  uint32_t* flag_bits = nullptr;   // [flag_words(T_ant cells)] bit e: entry e has valid == 2
  int32_t* n_flag = nullptr;       // [1] number of ill-conditioned entries
  int64_t* flag_list = nullptr;    // [T_ant cells] their indices, ascending
  // rect
  float4* pa = nullptr;          // [T_ant][N+1][2] FP64 antenna prefix (a2, b2, ab, 0) as hi4, lo4
  float4* px = nullptr;          // [T][N+1][2] float-float data prefix (hi4, lo4)
  // exp: chunk-major copies of the atoms (perm_entries(N, lanes) per set)
  // refinement: per-template fast statistics, histogram, chosen cut, the
  // candidates (cell, fast 2F, FP64 2F) and the plan's own map (if any)
  TStat* tstat = nullptr;        // [T]
  int32_t* ref_hist = nullptr;   // [T][kRefBins]
  int32_t* ref_ntile = nullptr;  // [T] tiles selected for the cell scan
  int32_t* ref_tile = nullptr;   // [T][kRefMaxTiles] their partial slots
  int32_t* ref_bin = nullptr;    // [T] last bin whose cells all lie in the scanned tiles
  int32_t* ref_n = nullptr;      // [T] candidates
  int32_t* ref_ncand = nullptr;  // [T] cells kept by the histogram pass (more than kRefCandCap: overflow)
  int32_t* ref_cand = nullptr;   // [T][kRefCandCap] those cells
  int32_t* ref_cell = nullptr;   // [T][kRefMaxCells]
  float* ref_fast = nullptr;     // [T][kRefMaxCells]
  double* ref_val = nullptr;     // [T][kRefMaxCells] (-1: invalid in FP64)
  float* own_map = nullptr;      // [T][cells] (FMAP_PLAN_MAP_BUFFER)
  float4* perm_ant = nullptr;    // [T_ant][.] (a2, b2, ab, gap to the next atom as int bits; -1 last)
  float4* perm_x = nullptr;      // [T][.] (Fa re, Fa im, Fb re, Fb im); recurrence plans
  int32_t* perm_gap = nullptr;   // [.] gap to the next atom (-1 last); recurrence plans
  // recurrence plans: per cell, tau-major ([n_tau][n_t0]), the window record
  // (i0, j as int bits, prefactor, tail factor), then a copy of the
  // coefficients (shared antenna): written by the recurrence kernel's first
  // template, read by the rest (absent with one template)
  float4* rec_cells = nullptr;   // [2][cells]
  // recurrence plans with two or more templates: the FP32 decay after each
  // atom, per tau in the chunk-major order (first template writes, the rest
  // read)
  float* rec_decay = nullptr;    // [n_tau][perm_entries]
  TauTab* tauc = nullptr;        // [n_tau] per-tau decay constants
  float2* wtab = nullptr;        // table windows: [kTabMax + 1] (w_k, w_{k+1} - w_k), then (0, 0)
  int64_t* ax = nullptr;         // [n_t0 + n_tau] explicit axes: t0 values, then tau values
  // exp
  float2* esuf = nullptr;        // [tau_chunk][3][N+1] float-float decayed suffix sums
  // tensor-core operands
  void* xop = nullptr;           // split X operands (layout per precision)
  // host-API staging
  int64_t* st_t = nullptr;
  float* st_ant = nullptr;
  float* st_x = nullptr;
  float* st_map = nullptr;
  fmap_summary* st_sum = nullptr;
};

}  // namespace fmap

struct fmap_plan_s {
  fmap_grid grid;
  int32_t n_sft = 0;
  int32_t n_templates = 0;
  fmap_precision precision = FMAP_FP64;
  uint32_t flags = 0;
  double log_prior = 0.0;
  int32_t refine_cells = -1;  // fmap_plan_set_refine (< 0: the precision's default)
  fmap::TileGeom tiles{};      // reduction tiles of the last compute call's main kernel
  int64_t wait_ns = fmap::kDefaultWaitNs;   // fmap_plan_set_wait_limit
  int device = 0;
  int n_sm = 0;
  int64_t n_tiles = 0;        // partial slots per template of the main kernels
  int64_t part_stride = 0;    // n_tiles + kFixSlots
  int32_t tau_chunk = 0;      // exp: tau values per suffix launch
  size_t xop_bytes = 0;
  bool host_staging = false;
  // explicit (t0, tau) axes set by fmap_plan_axes (in ws.ax; else the uniform
  // grid of Eq. Fmn); host copy of the axes
  bool explicit_axes = false;
  std::vector<int64_t> ax_host;
  int32_t n_tab = 0;             // table windows: samples set by fmap_plan_window_table
  int32_t lanes = fmap::kScanLanes;   // exp scan width (threads per tau)
  // TMA descriptors (CUtensorMap, 128 bytes each) of the split X operands
  alignas(64) unsigned char tmap_hi[128] = {};
  alignas(64) unsigned char tmap_lo[128] = {};
  bool tmaps_ready = false;
  bool owns_ws = false;          // workspace allocated by fmap_plan (else caller-provided)
  bool needs_err_reset = true;   // status word not yet cleared on the device
  // FMAP_PLAN_GRAPH: the captured call, the pointers it was captured with
  // (atoms t, antenna, fafb, shared flag, map, summaries, window) and its
  // launch count
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;   // where the graph was last launched
  const void* graph_key[6] = {};
  int32_t graph_key_window = -1;
  int64_t graph_launches = 0;
  cudaStream_t last_stream = nullptr;
  fmap::Workspace ws;
  // timing (fmap_plan_enable_timing)
  bool timing = false;
  int64_t launches = 0;       // kernels launched since timing was enabled
  std::vector<cudaEvent_t> events;  // FMAP_N_PHASES + 1 per timed call
};

namespace fmap {

// The explicit axes of a plan for its kernels, or null for a uniform grid.
inline const int64_t* plan_axes(const fmap_plan_s* p) { return p->explicit_axes ? p->ws.ax : nullptr; }

// ---- host launchers (each returns cudaGetLastError of its launches and
// adds the number of kernels it launched to p->launches) -------------------
cudaError_t launch_prep(fmap_plan_s* p, const fmap_atoms* a, cudaStream_t s);
cudaError_t launch_index(fmap_plan_s* p, const int64_t* d_t, cudaStream_t s);
// Each compute launcher reports how many partial slots per template it wrote.
// launch_rect records `mark` (if non-null) between its prefix scans and the
// per-cell kernel.
cudaError_t launch_rect(fmap_plan_s* p, const fmap_atoms* a, float* d_2F, cudaStream_t s,
                        int64_t* tiles_used, cudaEvent_t mark);
cudaError_t launch_exp_coef(fmap_plan_s* p, const fmap_atoms* a, cudaStream_t s);
cudaError_t launch_exp_perm(fmap_plan_s* p, const fmap_atoms* a, cudaStream_t s);
cudaError_t launch_table_antenna(fmap_plan_s* p, const fmap_atoms* a, cudaStream_t s);
cudaError_t launch_exp_plain(fmap_plan_s* p, const fmap_atoms* a, float* d_2F, cudaStream_t s,
                             int64_t* tiles_used);
cudaError_t launch_exp_tc(fmap_plan_s* p, const fmap_atoms* a, float* d_2F, cudaStream_t s,
                          int64_t* tiles_used);
cudaError_t launch_exp_rec(fmap_plan_s* p, const fmap_atoms* a, float* d_2F, cudaStream_t s,
                           int64_t* tiles_used);
bool exp_rec_supported(int32_t n_sft, int32_t n_t0);
bool exp_antenna_fits(int32_t n_sft);
size_t exp_antenna_smem(int32_t n_sft);
// Dynamic shared memory of the recurrence for blocks of up to tpb templates.
size_t exp_rec_smem(int32_t n_sft, int32_t n_t0, int32_t tpb);
// Dispatcher kernels of the batch phases, by file (nullptr: not that file's).
const void* batch_kernel_common(int phase);
const void* batch_kernel_rect(int phase);
// The exp scan phases have one dispatcher per scan width.
const void* batch_kernel_exp(int phase, int lanes);
const void* batch_kernel_exp_rec(int phase, int lanes);
const void* batch_kernel_fixup(int phase);
cudaError_t launch_rect_coef(fmap_plan_s* p, const fmap_atoms* a, cudaStream_t s);
cudaError_t launch_flag_and_fixup(fmap_plan_s* p, const fmap_atoms* a, float* d_2F,
                                  cudaStream_t s);
// Top-cell refinement of the summaries (after launch_final_reduce); d_2F is
// the map the compute call wrote, n_tiles the main kernel's partial slots
// (geometry p->tiles).
cudaError_t launch_refine(fmap_plan_s* p, const fmap_atoms* a, float* d_2F,
                          fmap_summary* d_summary, int64_t n_tiles, cudaStream_t s);
// Candidates per template of a plan's refinement (0: off).
int32_t refine_cells_of(const fmap_plan_s* p);
// Reduces partial slots [0, n_tiles) and, when with_fix, the fix-up slots.
cudaError_t launch_final_reduce(fmap_plan_s* p, int64_t n_tiles, bool with_fix,
                                fmap_summary* d_summary, cudaStream_t s);
cudaError_t launch_marginalise(fmap_plan_s* p, const float* d_2F, const uint8_t* d_valid,
                               fmap_summary* d_summary, cudaStream_t s);
// Marginalisation with caller-provided partial storage: marg_tiles(g) slots
// per template, packed ([T][marg_tiles(g)]).
cudaError_t launch_marginalise_into(const fmap_grid& g, int32_t n_templates, const float* d_2F,
                                    const uint8_t* d_valid, Partial* parts, double log_prior,
                                    fmap_summary* d_summary, cudaStream_t s);
bool grid_is_valid(const fmap_grid* g, std::string* why);
// Plans in caller-provided workspace (used by the server): the footprint,
// initialisation without allocation, and release of what a plan holds besides
// its workspace.
fmap_status plan_footprint(const fmap_grid* grid, int32_t n_sft, int32_t n_templates,
                           fmap_precision precision, uint32_t flags, size_t* bytes);
fmap_status plan_init(fmap_plan_s* p, const fmap_grid* grid, int32_t n_sft, int32_t n_templates,
                      fmap_precision precision, uint32_t flags, void* base, size_t bytes);
void plan_release(fmap_plan_s* p);

// First-level groups of the final reduction for `slots` partials.
int64_t reduce_groups_of(int64_t slots);
constexpr size_t kGroupBytes = 32;

// Entries of the padded relative-time array.
inline int32_t rel_t_entries(int32_t n_sft) { return ((n_sft + 63) / 64) * 64 + 64; }

// Tile counts of each kernel family (partials per template).
int64_t rect_tiles(const fmap_grid& g);
// y extent of the fix-up grid (kFixSlots x this) for a template count.
int64_t fixup_blocks_y(int32_t n_templates);
// The rectangular cells phase: partial slots per template, blocks and
// dynamic shared memory of its kernel.
int64_t rect_partial_slots(const fmap_grid& g, int32_t n_templates, int32_t shared_antenna);
int64_t rect_cells_blocks(const fmap_grid& g, int32_t n_templates, int32_t shared_antenna);
size_t rect_cells_smem(int32_t n_templates, int32_t shared_antenna);
int64_t exp_tiles(const fmap_grid& g);
int64_t marg_tiles(const fmap_grid& g);
bool exp_tc_available(fmap_precision prec);
size_t exp_tc_operand_bytes(const fmap_grid& g, int32_t n_sft, int32_t n_templates,
                            fmap_precision prec);

}  // namespace fmap
