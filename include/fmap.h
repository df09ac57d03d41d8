/*
 * fmap -- transient F-statistic maps on one GB300 (sm_103a).
 *
 * C ABI of libfmap.so.  The operation (Keitel & Ashton, arXiv:1805.05652):
 * from per-SFT atoms {a^2, b^2, ab, Fa, Fb} (Sec. 2 after Eq. F_xMx; Sec. 3
 * sends them to the GPU as a 7 x N_SFT real matrix) compute, for every cell
 * (t0_m, tau_n) of a uniform grid (Eq. Fmn), the windowed sums
 *   A = sum w^2 a^2, B = sum w^2 b^2, C = sum w^2 ab, Fa = sum w Fa_a,
 *   Fb = sum w Fb_a
 * with the rectangular window of Eq. (winrect) or the exponential window of
 * Eq. (winexp) (cut after 3 tau by default), the determinant D = A B - C^2 and
 * 2F from Eq. (F_FaFb); fused with the per-template reductions max 2F,
 * argmax (m, n) and the log Bayes factor marginalised over (t0, tau)
 * (Sec. 2 Eq. F_OSG; App. A).
 *
 * Conventions shared by every entry point:
 *   - Times are integer seconds (int64).  An SFT that starts at t is inside the
 *     window of (t0, tau) when t0 <= t and t + T_sft <= t0 + L, L = tau (rect)
 *     or L = 3 tau (exp; exp_cut8 / 8 tau in general).  Windows past the end of the data are truncated
 *     (App. A, non-embedded convention).
 *   - A cell with fewer than 2 SFTs in its window (Sec. 4.1) or with D <= 0
 *     is invalid: its 2F is 0 and it is left out of max, argmax and logB.
 *   - logB = ln((1/N_valid) sum_valid e^{2F/2}) + log_prior_const.
 *   - argmax ties go to the lowest m * n_tau + n.
 *   - Device buffers are caller-owned plain device pointers; the plan owns
 *     its workspace.  Compute calls are asynchronous on the given stream and
 *     never throw; errors are status codes.  Data errors found on the device
 *     (non-increasing timestamps, a time span >= 2^31 s) are latched in the
 *     plan and returned by fmap_plan_status(); so are non-finite atoms
 *     (FMAP_ERR_NONFINITE), which leave that call's outputs undefined.
 *   - A plan serialises its own calls: do not use one plan from two host
 *     threads at once, nor on two streams whose work overlaps.
 */
#ifndef FMAP_H
#define FMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; 0 is the legacy default stream. */
typedef struct CUstream_st* fmap_stream;

typedef enum {
  FMAP_OK = 0,
  FMAP_PENDING = 1,          /* fmap_poll: not finished yet */
  FMAP_ERR_ARG = -1,         /* invalid argument (sizes, grid, null pointer) */
  FMAP_ERR_NOMEM = -2,       /* device or host allocation failed / over budget */
  FMAP_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  FMAP_ERR_TIMEOUT = -4,     /* a bounded wait gave up */
  FMAP_ERR_BUSY = -5,        /* server full / ticket unknown */
  FMAP_ERR_DATA = -6,        /* timestamps not strictly increasing or span >= 2^31 s */
  FMAP_ERR_UNSUPPORTED = -7, /* valid request outside what the library supports */
  FMAP_ERR_NONFINITE = -8    /* an atom (antenna or data row) is NaN or infinite */
} fmap_status;

/* FMAP_TABLE: a generic window function w(x), x = (t - t0) / tau, given as a
 * table of samples (fmap_plan_window_table), on the exponential window's
 * support [t0, t0 + floor(exp_cut8 tau / 8)]. */
typedef enum { FMAP_RECT = 0, FMAP_EXP = 1, FMAP_TABLE = 2 } fmap_window;

/*
 * Arithmetic of the windowed sums.  In every mode the antenna sums A, B, C
 * and the determinant D = AB - C^2 are float-float (pairs of FP32 numbers
 * with error-free FMA products, ~2^-44 relative: GB300 runs FP64 at 1/64 of
 * the FP32 rate), the 2F coefficients FP32 from them (once per cell), and
 * the log-Bayes reduction FP64:
 *   FMAP_FP64   rect: FP64 prefix sums over SFTs (data rows kept as float
 *               pairs), O(1) compensated differences per cell;
 *               exp:  FP64 contraction on the CUDA cores.
 *   FMAP_FP32   rect: one thread per t0 row with FP32 running sums of Fa, Fb
 *               (the paper's rectangular kernel, Sec. 3);
 *               exp:  FP32 contraction on the CUDA cores (the plain path).
 *   FMAP_TF32   exp only: tensor-core contraction (tcgen05, kind::tf32) with
 *               both operands split hi + lo, three products, FP32 accumulate.
 *   FMAP_BF16X3 exp only: tensor-core contraction (tcgen05, kind::f16, bf16)
 *               with hi*hi + hi*lo + lo*hi, FP32 accumulate.
 * Cells whose antenna matrix is ill-conditioned (A B / D > 100: windows of a
 * few SFTs of one detector, where any FP32 sum loses ~1e-7 sqrt(AB/D) of
 * relative accuracy in 2F) are recomputed from their atoms in every mode:
 * windowed sums, D and the numerator of 2F in float-float (~2^-46 A B / D
 * relative), one FP32 quotient.
 */
typedef enum { FMAP_FP64 = 0, FMAP_FP32 = 1, FMAP_TF32 = 2, FMAP_BF16X3 = 3 } fmap_precision;

/* Grid of Eq. (Fmn): t0_m = t0_min + m dt0 (m < n_t0), tau_n = tau_min + n dtau
 * (n < n_tau).  Needs n_t0, n_tau >= 0, tau_min > 0, t_sft > 0, dtau > 0 when
 * n_tau > 1, dt0 > 0 when n_t0 > 1, L(tau_max) < 2^31.
 * exp_cut8: length of the exponential window in eighths of tau, L(tau) =
 * floor(exp_cut8 tau / 8) seconds (Eq. winexp is cut after 3 tau: 0 selects
 * the default 24; 1..1024 allowed); ignored for rect windows (L = tau).  It
 * sits in what was padding, so a zero-initialised grid keeps the 3 tau cut. */
typedef struct {
  int64_t t0_min;
  int64_t dt0;
  int32_t n_t0;
  int64_t tau_min;
  int64_t dtau;
  int32_t n_tau;
  int64_t t_sft;
  int32_t window;   /* fmap_window */
  int32_t exp_cut8; /* exp window length in tau / 8 (0: 24, i.e. 3 tau) */
} fmap_grid;

/* Atoms (Sec. 3: 3 real rows a^2, b^2, ab and 2 complex rows Fa, Fb).
 * t        [n_sft] int64, strictly increasing SFT start times;
 * antenna  [3][n_sft] float (a^2, b^2, ab) if shared_antenna, else [T][3][n_sft];
 * fafb     [T][4][n_sft] float (Re Fa, Im Fa, Re Fb, Im Fb).
 * Device pointers for fmap_compute_*, host pointers for fmap_compute_host and
 * fmap_submit.  Rows need no alignment beyond 4 bytes. */
typedef struct {
  int32_t n_sft;
  int32_t n_templates;
  int32_t shared_antenna;
  const int64_t* t;
  const float* antenna;
  const float* fafb;
} fmap_atoms;

/* Per-template result (32 bytes).  n_valid = 0 gives max2F = 0, m = n = -1,
 * logB = NaN.  flags: FMAP_SUMMARY_* bits (see fmap_plan_set_refine). */
typedef struct {
  float max2F;
  int32_t m;
  int32_t n;
  int32_t flags;
  double logB;
  int64_t n_valid;
} fmap_summary;

enum {
  /* the cells nearest the maximum were recomputed from their atoms
   * (float-float window sums, D and 2F in FP64) and max2F, the argmax and
   * logB use those values */
  FMAP_SUMMARY_REFINED = 1u,
  /* every cell whose fast 2F lay within the fast path's error bound of the
   * maximum was among them: the argmax was decided on FP64 values */
  FMAP_SUMMARY_ARGMAX_EXACT = 2u
};

/* fmap_plan flags */
enum {
  /* atoms carry antenna rows per template ([T][3][n_sft]); workspace for the
   * per-template 2F coefficients grows by a factor T */
  FMAP_PLAN_PER_TEMPLATE_ANTENNA = 1u,
  /* exponential windows only, with FMAP_FP64: the data sums by the decayed
   * suffix recurrence E[i] = x_i + e^{-(t_{i+1} - t_i)/tau} E[i+1] (an exact
   * rearrangement of Eq. winexp's window sums: window [i0, j) =
   * e^{-(t_i0 - t0)/tau} (E[i0] - e^{-(t_j - t_i0)/tau} E[j])), one scan per
   * (tau, data column) in compensated FP32 instead of a sum per cell:
   * O(N_tau N_SFT + cells) per template.  Needs n_sft <= 9000 (one
   * template's suffix sums in shared memory; FMAP_ERR_UNSUPPORTED otherwise);
   * with two or more templates the workspace also holds the per-cell window
   * records and per-atom decays of every tau (32 B per cell, 4 B per atom
   * and tau), formed by a block's first template and re-read by the rest. */
  FMAP_PLAN_EXP_RECURRENCE = 2u,
  /* the plan holds a [T][n_t0][n_tau] float map of its own (the workspace
   * grows by 4 T n_t0 n_tau bytes), used by summary-only compute calls
   * (d_2F = NULL) so that their summaries can be refined (fmap_plan_set_refine);
   * without it a summary-only call reports the unrefined reductions */
  FMAP_PLAN_MAP_BUFFER = 4u,
  /* repeated compute calls replay one CUDA graph of the call's launches: the
   * first call with a given set of atom, map and summary pointers captures
   * its launches (on a stream of the plan's own) and launches the graph on
   * the caller's stream; later calls with the same pointers launch it again
   * (the data behind the pointers may change between calls), other pointers
   * capture anew, and so does the first call after a setting of the plan
   * changes (log prior, refinement, wait limit, axes, window table).  Plans
   * with timing enabled launch directly. */
  FMAP_PLAN_GRAPH = 8u
};

typedef struct fmap_plan_s fmap_plan_t;
typedef struct fmap_server_s fmap_server_t;

/*
 * fmap_plan: create a plan for one grid, SFT count and template count
 * (the F-map problem statement of Sec. 3: atoms + window + grid).  The plan
 * allocates its workspace (fmap_workspace_bytes) on the current device.
 * flags: FMAP_PLAN_* bits.  Returns FMAP_ERR_ARG on an invalid grid or size,
 * FMAP_ERR_UNSUPPORTED for a precision the window does not offer,
 * FMAP_ERR_NOMEM when the workspace cannot be allocated.
 */
fmap_status fmap_plan(fmap_plan_t** plan, const fmap_grid* grid, int32_t n_sft,
                      int32_t n_templates, fmap_precision precision, uint32_t flags);
void fmap_plan_destroy(fmap_plan_t* plan);

/* Explicit (t0, tau) axes: a non-uniform or undersampled grid in place of
 * Eq. (Fmn)'s uniform steps.  t0_values [n_t0] and tau_values [n_tau] are
 * HOST arrays of strictly increasing integer seconds (tau > 0, the window
 * length at the largest tau < 2^31 s, t0 within +-2^62); they are copied into
 * the plan's workspace (synchronously, after the plan's last stream has
 * drained).  While set, the grid's t0_min, dt0, tau_min and dtau are unused;
 * n_t0, n_tau, t_sft, window and exp_cut8 still apply.  Both NULL restores the
 * uniform grid.  Errors: FMAP_ERR_ARG (one NULL, bad values), FMAP_ERR_CUDA.
 * Batches and the server take uniform grids only. */
fmap_status fmap_plan_axes(fmap_plan_t* plan, const int64_t* t0_values,
                           const int64_t* tau_values);
/* fmap_count_terms for a plan's grid (its explicit axes if set). */
fmap_status fmap_plan_count_terms(fmap_plan_t* plan, const int64_t* t, int32_t n_sft,
                                  int64_t* n_terms, int64_t* n_cells_2plus);

/* Workspace a plan of these sizes allocates (bytes). */
size_t fmap_workspace_bytes(const fmap_grid* grid, int32_t n_sft, int32_t n_templates,
                            fmap_precision precision);

/* Additive constant of logB (prior normalisation; default 0). */
fmap_status fmap_plan_set_log_prior(fmap_plan_t* plan, double log_prior_const);

/*
 * Refinement of the reductions (Sec. 2 Eq. F_OSG: the argmax is the
 * detection candidate and e^F the odds, so both are decided on FP64 values).
 * After a compute call's fast map and reductions, per template the cells
 * whose fast 2F lies within 16 of the fast maximum (at most max_cells of
 * them, the highest; a histogram of 256 bins picks the cut; when more than
 * max_cells lie within 1/16 of the maximum, all of those, up to 4096, else
 * none and the flags stay 0) are recomputed
 * from their atoms by the plain definition (windowed sums in float-float,
 * ~2^-44 relative; D and Eq. F_FaFb in FP64); these values replace the fast
 * ones in the map, in max2F, in the argmax (lowest index on ties) and in
 * logB (the fast exp-sum has their fast terms replaced by the refined
 * ones).  Summary flags:
 * FMAP_SUMMARY_REFINED once this ran, FMAP_SUMMARY_ARGMAX_EXACT when the cut
 * lies below the maximum by more than twice the precision's error bound
 * (1e-5 relative for FMAP_FP64, 1e-3 otherwise, floor 1), so that no other
 * cell can hold the maximum.  max_cells: 0 turns refinement off, < 0 selects
 * the default (64 for FMAP_FP64 plans, 512 otherwise), at most 4096.  Needs
 * the map: the caller's d_2F, else the plan's own (FMAP_PLAN_MAP_BUFFER).
 * Batches do not refine.
 */
fmap_status fmap_plan_set_refine(fmap_plan_t* plan, int32_t max_cells);

/*
 * Limit of every bounded device wait of the plan's kernels (mbarrier waits
 * on bulk copies and tensor-core stages), in nanoseconds; < 0 restores the
 * default of 2 s.  0 makes a wait give up as soon as its first poll finds
 * the stage incomplete.  A wait that gives up latches FMAP_ERR_TIMEOUT
 * (fmap_plan_status) and the kernel winds down: it issues no further copies,
 * waits (up to 2 s) for those already in flight, releases its tensor memory
 * and returns; that call's outputs are undefined.
 */
fmap_status fmap_plan_set_wait_limit(fmap_plan_t* plan, int64_t limit_ns);

/*
 * fmap_compute_rect / fmap_compute_exp: the F-map of Eq. (Fmn) for every
 * template with the rectangular (Eq. winrect) or exponential (Eq. winexp)
 * window; the grid's window field must match.  Sec. 3 (the two kernels, D
 * and F inside the GPU), Eq. (F_FaFb).
 *   atoms      device atoms, n_sft / n_templates equal to the plan's;
 *   d_2F       nullable device [T][n_t0][n_tau] float, 2F per cell (n fastest);
 *   d_summary  nullable device [T] fmap_summary.
 * Asynchronous on stream.  FMAP_ERR_ARG on mismatched sizes or window.
 */
fmap_status fmap_compute_rect(fmap_plan_t* plan, const fmap_atoms* atoms, float* d_2F,
                              fmap_summary* d_summary, fmap_stream stream);
fmap_status fmap_compute_exp(fmap_plan_t* plan, const fmap_atoms* atoms, float* d_2F,
                             fmap_summary* d_summary, fmap_stream stream);

/*
 * Generic window functions (FMAP_TABLE grids): the paper's windowed sums
 * with any amplitude envelope w in place of Eq. (winrect) / (winexp).
 * fmap_plan_window_table: w sampled at n_points (2..1024) equally spaced
 * x_k = k X / (n_points - 1), X = exp_cut8 / 8 (24 / 8 = 3 by default), as a
 * HOST float array, copied into the plan (synchronously); between samples w
 * is linear, beyond X it is 0.  The atom at t weighs w((t - t0) / tau) in Fa,
 * Fb and w^2 in A, B, C (membership as for exp windows).  Errors: FMAP_ERR_ARG
 * (not a table plan, bad size or non-finite values), FMAP_ERR_CUDA.
 * fmap_compute_table: as fmap_compute_exp for a table plan (FMAP_FP64 and
 * FMAP_FP32 on the CUDA cores, FMAP_TF32 and FMAP_BF16X3 on the tensor cores;
 * the antenna sums A, B, C are float-float sums over each window); the table
 * must be set first (else FMAP_ERR_ARG).  Batches and the server do not take
 * table windows.
 */
fmap_status fmap_plan_window_table(fmap_plan_t* plan, const float* w, int32_t n_points);
fmap_status fmap_compute_table(fmap_plan_t* plan, const fmap_atoms* atoms, float* d_2F,
                               fmap_summary* d_summary, fmap_stream stream);

/*
 * fmap_marginalise: the reductions alone (max 2F, argmax, marginalised logB;
 * Sec. 2 Eq. F_OSG, App. A) over a given map.
 *   d_2F      device [T][n_t0][n_tau] float (T = the plan's template count);
 *   d_valid   nullable device [T][n_t0][n_tau] uint8 (nonzero = valid); NULL
 *             treats every cell as valid;
 *   d_summary device [T].
 */
fmap_status fmap_marginalise(fmap_plan_t* plan, const float* d_2F, const uint8_t* d_valid,
                             fmap_summary* d_summary, fmap_stream stream);

/*
 * fmap_marginalise_noalloc: fmap_marginalise without a plan and without any
 * device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory once they are running -- a
 * latency-bound serving loop (cudaMalloc/cudaFree may synchronise the device
 * and take milliseconds) or a host application whose own allocator owns all
 * device memory.  Its reduction scratch is a fixed 8 MiB array inside the
 * library (fmap_noalloc_scratch_bytes()), held by every GPU that loads the
 * library until the process exits.  Limit: about 16 bytes per template and
 * 2048 cells (n_templates * ceil(n_t0 * n_tau / 2048) * 16 bytes plus a
 * small second-level area within 8 MiB, ~500k template-tiles), else
 * FMAP_ERR_ARG with a message.
 * The first call on each device (with that device current) looks up the
 * array's device address; make it before any stream capture.  After
 * cudaDeviceReset (which unloads the library's device code) the next call
 * looks the address up again: make that call outside stream capture too.
 * All calls
 * share the array, so calls whose work overlaps on the GPU race: serialise
 * them.  Nothing in the array needs clearing between calls.
 *   grid      the map's grid (window field unused); d_2F [T][n_t0][n_tau];
 *   d_valid   nullable [T][n_t0][n_tau] uint8, NULL = every cell valid;
 *   d_summary device [T]; asynchronous on stream.
 */
fmap_status fmap_marginalise_noalloc(const fmap_grid* grid, int32_t n_templates,
                                     const float* d_2F, const uint8_t* d_valid,
                                     double log_prior_const, fmap_summary* d_summary,
                                     fmap_stream stream);
size_t fmap_noalloc_scratch_bytes(void);

/*
 * fmap_compute_host: one synchronous end-to-end call with HOST buffers:
 * copies the atoms to plan-owned device staging (pinned host memory makes
 * the copies asynchronous), runs the window's compute, copies the map
 * (nullable h_2F) and the summaries (nullable h_summary) back, and waits.
 * The staging is allocated on the first call (the map's on the first call
 * that asks for the map); a summary-only call refines its summaries when the
 * plan has FMAP_PLAN_MAP_BUFFER.
 */
fmap_status fmap_compute_host(fmap_plan_t* plan, const fmap_atoms* host_atoms, float* h_2F,
                              fmap_summary* h_summary, fmap_stream stream);

/* Per-phase device timing of a plan's compute calls, taken with CUDA events
 * recorded on each call's stream.  Phases (FMAP_N_PHASES):
 *   0 input checks and window index tables,
 *   1 antenna sums / prefix sums (rect: FP64 scans; exp: float-float suffix
 *     sums and the per-cell 2F coefficients),
 *   2 the windowed contraction with the fused 2F epilogue (the dominant
 *     kernel),
 *   3 the recomputation of ill-conditioned cells, the final per-template
 *     reduction and the refinement of the summaries.
 * fmap_plan_enable_timing(plan, 1) starts recording (and clears the totals);
 * fmap_plan_read_timing waits for the recorded calls and returns the summed
 * milliseconds per phase, the number of timed calls and the number of
 * kernels the plan launched since timing was enabled. */
#define FMAP_N_PHASES 4
fmap_status fmap_plan_enable_timing(fmap_plan_t* plan, int32_t enable);
fmap_status fmap_plan_read_timing(fmap_plan_t* plan, double* ms, int64_t* calls,
                                  int64_t* launches);

/* Waits for the plan's last stream and returns (then clears) a latched data
 * or CUDA error, else FMAP_OK. */
fmap_status fmap_plan_status(fmap_plan_t* plan);

/*
 * Serving (continuous batching of F-map requests).  A server owns a device
 * memory pool of device_mem_budget bytes and a pinned host arena of
 * pinned_bytes, both allocated once by fmap_server_create, and a worker
 * thread.  fmap_submit copies a request's HOST atoms into the pinned arena
 * and queues it (the caller's buffers can be reused at once).  The worker
 * admits queued requests in arrival order whenever one of max_inflight
 * stream slots is free and the request's device footprint (plan workspace,
 * atoms, outputs) fits in the pool; each admitted request runs on its own
 * stream, so requests arriving while others are on the GPU overlap with
 * them.  A request's results do not depend on what else is in flight.
 * Precisions: rect_precision for rectangular windows; exponential windows
 * by exp_mode: FMAP_SERVER_EXP_FIXED takes exp_precision,
 * FMAP_SERVER_EXP_RECURRENCE the FP64-class decayed-suffix recurrence
 * (FMAP_FP64 with FMAP_PLAN_EXP_RECURRENCE), FMAP_SERVER_EXP_AUTO per request
 * whichever of the two a cost model of the form of App. A's timing model
 * (terms in N_SFT N_tau, N_sums and N_t0 N_tau per template, constants fitted
 * on GB300) estimates faster -- never less accurate than exp_precision
 * (data sets past the recurrence's 9000 SFTs take exp_precision).
 * Requests whose estimated GPU time is below 1 ms run on high-priority
 * streams, so their blocks are scheduled ahead of those still waiting from
 * larger requests in flight (the results do not change).
 * The paper computes one F-map per template on demand (Sec. 3, Sec. 4.2);
 * the server is the request loop around that operation.
 */
typedef struct {
  size_t device_mem_budget;
  size_t pinned_bytes;
  int32_t max_inflight;        /* 1..64 */
  fmap_precision exp_precision;
  fmap_precision rect_precision;
  uint32_t exp_mode;           /* FMAP_SERVER_EXP_* */
} fmap_server_config;
enum {
  FMAP_SERVER_EXP_FIXED = 0,
  FMAP_SERVER_EXP_RECURRENCE = 1,
  FMAP_SERVER_EXP_AUTO = 2
};

/* fmap_submit flags */
enum { FMAP_SUBMIT_MAP = 1u /* also return the 2F map */ };

fmap_status fmap_server_create(fmap_server_t** server, const fmap_server_config* config);
/* Stops the worker after the running requests finish; frees everything. */
void fmap_server_destroy(fmap_server_t* server);
/* grid: the request's grid (its window selects the path); host_atoms: HOST
 * pointers.  Returns a ticket.  FMAP_ERR_BUSY when the pinned arena is full
 * (poll finished requests, then resubmit); FMAP_ERR_NOMEM when the request
 * alone exceeds the device pool; FMAP_ERR_ARG / FMAP_ERR_UNSUPPORTED as
 * fmap_plan. */
fmap_status fmap_submit(fmap_server_t* server, const fmap_grid* grid,
                        const fmap_atoms* host_atoms, uint32_t flags, uint64_t* ticket);
/* Waits up to wait_us microseconds (0: no wait, < 0: until done) for a
 * ticket.  FMAP_PENDING: not finished.  Otherwise the request's status; on
 * FMAP_OK copies the summaries (h_summary, [T], nullable) and, if submitted
 * with FMAP_SUBMIT_MAP, the map (h_2F, [T][n_t0][n_tau], nullable).  A
 * finished ticket is released by this call; FMAP_ERR_BUSY for an unknown
 * ticket. */
fmap_status fmap_poll(fmap_server_t* server, uint64_t ticket, fmap_summary* h_summary,
                      float* h_2F, int64_t wait_us);
fmap_status fmap_server_stats(fmap_server_t* server, int64_t* queued, int64_t* running,
                              int64_t* completed);
/* The most requests that were running at once (on the GPU together) since
 * the server was created. */
fmap_status fmap_server_peak(fmap_server_t* server, int64_t* peak_running);

/*
 * Uneven batches: many independent F-map instances (each with its own atoms,
 * grid, window and template count; Sec. 3's per-template F-map, batched) run
 * by one captured CUDA graph.  Rectangular instances use the FP64 prefix
 * path, exponential ones the decayed-suffix recurrence (FMAP_FP64 accuracy
 * class, n_sft <= 9000).  Each phase of the pipeline is one persistent launch
 * over the work units of all instances (atomic work counter, heaviest
 * instances first); instances are grouped in waves whose workspace fits
 * workspace_budget (0: 8 GiB).  FMAP_BATCH_AUTOTUNE times the candidate
 * occupancies of each phase and the templates per block of the recurrence on
 * the batch itself (cached per batch shape) before the graph is captured.
 * The items' device pointers are baked into the graph: keep them valid, and
 * rerun fmap_batch_run after changing the atoms' values in place.
 */
typedef struct {
  fmap_grid grid;
  fmap_atoms atoms;          /* device pointers */
  float* d_2F;               /* nullable [T][n_t0][n_tau] */
  fmap_summary* d_summary;   /* nullable [T] */
} fmap_batch_item;

enum { FMAP_BATCH_AUTOTUNE = 1u };

typedef struct fmap_batch_s fmap_batch_t;

fmap_status fmap_batch_plan(fmap_batch_t** batch, const fmap_batch_item* items, int32_t n_items,
                            size_t workspace_budget, uint32_t flags);
/* Launches the batch's graph on stream (asynchronous). */
fmap_status fmap_batch_run(fmap_batch_t* batch, fmap_stream stream);
/* Waits for stream; returns (then clears) a latched data error or timeout of
 * any instance. */
fmap_status fmap_batch_status(fmap_batch_t* batch, fmap_stream stream);
/* Phases of a batch run, in launch order (FMAP_BATCH_N_PHASES entries):
 * input checks, index tables, exp chunk-major atom copies, rect antenna
 * prefixes, exp antenna sums and coefficients, rect coefficients, rect data
 * prefixes, exp recurrence and cells, rect cells, three steps of the
 * ill-conditioned cell compaction, float-float fix-up, two reduction levels. */
#define FMAP_BATCH_N_PHASES 15
/* Waves, kernel launches per run, workspace bytes, chosen occupancy per phase
 * (FMAP_BATCH_N_PHASES entries, nullable) and templates per block of the
 * recurrence. */
fmap_status fmap_batch_info(fmap_batch_t* batch, int32_t* n_waves, int64_t* launches_per_run,
                            size_t* workspace_bytes, int32_t* occupancy,
                            int32_t* rec_templates_per_block);
/* Profiling: runs the batch once phase by phase on stream (the same launches
 * as fmap_batch_run, outside the graph), times each with events and ADDS the
 * device milliseconds of each phase, summed over waves, to phase_ms
 * (FMAP_BATCH_N_PHASES entries).  Synchronous; writes the same outputs as a
 * run; must not overlap a run of the same batch (they share work counters). */
fmap_status fmap_batch_profile(fmap_batch_t* batch, fmap_stream stream, float* phase_ms);
void fmap_batch_destroy(fmap_batch_t* batch);

/*
 * Combining summaries of an F-map split by t0 rows (templates and t0 rows are
 * independent pieces of the map, Sec. 3): shard r computed rows
 * [m_offsets[r], m_offsets[r] + its n_t0) of every template and holds
 * summaries [n_shards][n_templates] (HOST arrays), m in its own rows.  Per
 * template: n_valid adds; max2F is the maximum over shards with valid cells
 * and the argmax the lowest global (m, n) attaining it; logB =
 * logsumexp_r(logB_r + ln N_r) - ln N (the shards' common prior constant
 * rides along); flags are those common to the non-empty shards.  Empty
 * shards (n_valid = 0) are skipped; all empty gives the empty summary
 * (max2F = 0, m = n = -1, logB = NaN).  Host only, exact up to FP64
 * rounding.  FMAP_ERR_ARG on NULL pointers or negative counts.
 */
fmap_status fmap_combine_summaries(const fmap_summary* shards, int32_t n_shards,
                                   int32_t n_templates, const int32_t* m_offsets,
                                   fmap_summary* out);

/* Host-side window bookkeeping for throughput accounting: over all cells,
 * the total number of (cell, SFT) terms (sum of atoms per window, App. A
 * Eq. Nsums-exp for exp windows) and the number of cells with >= 2 atoms.
 * t is a HOST pointer. */
fmap_status fmap_count_terms(const fmap_grid* grid, const int64_t* t, int32_t n_sft,
                             int64_t* n_terms, int64_t* n_cells_2plus);

const char* fmap_status_string(fmap_status status);
/* Message of the last error on this host thread ("" if none). */
const char* fmap_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FMAP_H */
