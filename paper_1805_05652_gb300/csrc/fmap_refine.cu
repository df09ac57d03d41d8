// Top-cell refinement of the per-template reductions.
//
// The detection statistic of a template is its maximum 2F and the cell that
// holds it, and e^F is the odds of a transient in that cell (Sec. 2, Eq.
// F_OSG), so the marginalised Bayes factor is dominated by the cells nearest
// the maximum.  After a compute call has written its fast map, reduced it
// (max, argmax, exp-sum, count) and recomputed the ill-conditioned cells,
// this stage, per template:
//   1. histograms the valid cells whose fast 2F lies within kRefWindow of the
//      fast maximum M (kRefBins bins, bin 0 at the maximum) -- reading only
//      the tiles whose fast maximum (from the reduction partials) can bound
//      one of the cells the cut will take, so the cost does not grow with
//      the map;
//   2. cuts the histogram after the last bin that keeps the cell count within
//      the plan's cap (or after the top bin, when it alone holds more, up to
//      kRefMaxCells), and collects those cells (in no fixed order: every
//      later reduction over them is order-independent -- integer sums of
//      fixed-point terms and a minimum of cell indices): from the cells the
//      histogram pass kept (those in bins up to the tile pass's bound, at
//      most kRefCandCap per template), else by a second scan of the tiles;
//   3. recomputes each collected cell from its atoms by the plain
//      definition: the windowed sums of Eq. (winrect) / (winexp) with w on
//      Fa, Fb and w^2 on A, B, C (in float-float, ~2^-44 relative), then
//      D = AB - C^2 and 2F of Eq. (F_FaFb) in FP64; the refined value
//      replaces the fast one in the map;
//   4. rebuilds the summary: max2F and the argmax (lowest index on FP64
//      ties) from the FP64 values, and the exp-sum with the collected cells'
//      fast terms replaced by their FP64 terms,
//        S' = e^{(M - M')/2} (S - sum_k e^{(f_k - M)/2}) + sum_k e^{(v_k - M')/2},
//      logB = M'/2 + ln S' - ln N' + c.
// Every cell outside the cut had a fast 2F more than the cut's distance d
// below M; when d exceeds twice the fast path's error bound, no such cell
// can hold the FP64 maximum, and the summary says so (ARGMAX_EXACT).
#include <math.h>

#include "fmap_device.cuh"

namespace fmap {

constexpr int kRefThreads = 256;
constexpr int kScanShare = 256;   // cells of a listed tile per scanning warp

int32_t refine_cells_of(const fmap_plan_s* p) {
  if (p->refine_cells == 0 || !p->ws.tstat) return 0;
  if (p->refine_cells > 0) return std::min(p->refine_cells, kRefMaxCells);
  return p->precision == FMAP_FP64 ? 64 : 512;
}

// Relative error bound (floor 1) of a plan's fast 2F.
static double fast_tol(const fmap_plan_s* p) { return p->precision == FMAP_FP64 ? 1e-5 : 1e-3; }

// Coef.valid of cell c for template j: 1 summed by the main kernel, 3
// recomputed by the fix-up (and summed in a fix-up slot), else invalid.
__device__ __forceinline__ float ref_valid_of(const Coef* __restrict__ coef, int32_t shared,
                                              int64_t cells, int32_t j, int64_t c) {
  return coef[shared ? c : (int64_t)j * cells + c].valid;
}

// Bin of a fast value v against the template's maximum M: floor((M - v)
// kRefBins / kRefWindow), -1 outside the window (or not a number).
__device__ __forceinline__ int ref_bin_of(float v, float M) {
  const float d = (M - v) * ((float)kRefBins / kRefWindow);
  if (!(d < (float)kRefBins)) return -1;
  return d > 0.0f ? (int)d : 0;
}

// The last histogram bin whose cumulative count stays within the cap, at
// most bt (the last bin whose cells all lie in scanned tiles).  When the top
// bin alone holds more than the cap (a maximum shared by many cells within
// 1/16 of 2F, e.g. windows truncated at the data's end), the top bin as a
// whole while it fits the candidate buffer; else -1 (no refinement).
__device__ __forceinline__ int32_t ref_cut_of(const int32_t* __restrict__ h, int32_t cap,
                                              int32_t bt) {
  int32_t cum = 0, b = -1;
  for (int k = 0; k <= bt && k < kRefBins; ++k) {
    cum += h[k];
    if (cum > cap) break;
    b = k;
  }
  if (b < 0 && h[0] <= kRefMaxCells) b = 0;
  return b;
}

// Pass 1 (one block per template): which tiles to scan.  The partials give
// every tile's fast maximum (a main tile's over the cells the main kernel
// summed, a fix-up slot's over its recomputed cells: disjoint sets); with bt
// the first bin in which the count of tiles (by their maxima) reaches the
// cap, at least cap distinct cells lie in bins <= bt (those maxima), so the
// cut never passes bt, and every cell in a bin <= bt lies in a tile whose
// maximum is in a bin <= bt: those tiles are listed for the cell passes,
// and bt is kept in cut[j].
constexpr int kTileThreads = 1024;
constexpr int kTileCache = 8;   // slots per thread whose bins stay in registers

__global__ void __launch_bounds__(kTileThreads)
k_ref_tiles(const Partial* __restrict__ parts, int64_t stride, int64_t n_tiles, int64_t fix0,
            int64_t n_fix, const TStat* __restrict__ st, int32_t cap,
            int32_t* __restrict__ ref_ntile, int32_t* __restrict__ ref_tile,
            int32_t* __restrict__ cut, int32_t* __restrict__ ref_ncand) {
  __shared__ int32_t h[kRefBins];
  __shared__ int32_t s_bt, s_n;
  const int32_t j = blockIdx.x;
  const int lane = threadIdx.x & 31;
  for (int b = threadIdx.x; b < kRefBins; b += blockDim.x) h[b] = 0;
  if (threadIdx.x == 0) {
    s_n = 0;
    ref_ncand[j] = 0;   // (the histogram pass after this one counts its kept cells)
  }
  __syncthreads();
  const TStat s = st[j];
  const Partial* pp = parts + (int64_t)j * stride;
  const int64_t total = s.N > 0 ? n_tiles + n_fix : 0;
  auto bin_of = [&](int64_t k) {
    if (k >= total) return -1;
    const Partial q = pp[k < n_tiles ? k : fix0 + (k - n_tiles)];
    return q.nvalid > 0 ? ref_bin_of(q.max2F, s.M) : -1;
  };
  // one shared-memory atomic per distinct bin among a warp's lanes
  auto count = [&](int b, unsigned mask) {
    const unsigned peers = __match_any_sync(mask, b);
    if (b >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h[b], __popc(peers));
  };
  int bins[kTileCache];
#pragma unroll
  for (int i = 0; i < kTileCache; ++i) {
    bins[i] = bin_of(threadIdx.x + (int64_t)i * kTileThreads);
    count(bins[i], 0xffffffffu);
  }
  for (int64_t k = threadIdx.x + (int64_t)kTileCache * kTileThreads; k < total; k += kTileThreads)
    count(bin_of(k), __activemask());
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t cum = 0, bt = kRefBins - 1;
    for (int k = 0; k < kRefBins; ++k) {
      cum += h[k];
      if (cum >= cap) {
        bt = k;
        break;
      }
    }
    s_bt = bt;
  }
  __syncthreads();
  const int32_t bt = s_bt;
  int32_t* list = ref_tile + (int64_t)j * kRefMaxTiles;
  auto put = [&](int64_t k, int b, unsigned mask) {
    const bool take = b >= 0 && b <= bt;
    const unsigned sel = __ballot_sync(mask, take);
    if (!sel) return;
    const int leader = __ffs(sel) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(&s_n, __popc(sel));
    base = __shfl_sync(mask, base, leader);
    const int32_t at = base + __popc(sel & ((1u << lane) - 1u));
    if (take && at < kRefMaxTiles) list[at] = (int32_t)k;
  };
#pragma unroll
  for (int i = 0; i < kTileCache; ++i)
    put(threadIdx.x + (int64_t)i * kTileThreads, bins[i], 0xffffffffu);
  for (int64_t k = threadIdx.x + (int64_t)kTileCache * kTileThreads; k < total; k += kTileThreads)
    put(k, bin_of(k), __activemask());
  __syncthreads();
  if (threadIdx.x == 0) {
    ref_ntile[j] = s_n;   // (more than kRefMaxTiles: truncated)
    cut[j] = bt;
  }
}

struct ScanArgs {
  const float* map;
  const Coef* coef;
  int32_t shared;
  int32_t n_t0, n_tau;
  int64_t cells;
  TileGeom geo;
  int64_t n_tiles;
  int32_t parts;   // warps per listed tile (each takes one share of its cells)
  const int64_t* flag_list;
  const int32_t* n_flag;
  int32_t n_templates;
  const TStat* st;
  const int32_t* ref_ntile;
  const int32_t* ref_tile;
  int32_t* hist;
  int32_t cap;
  const int32_t* cut;   // [T] bt of the tile pass
  int32_t* ref_n;
  int32_t* ref_cell;
  int32_t* ref_ncand;
  int32_t* ref_cand;
};

// Calls f(cell, owned) for every cell of share `part` (of A.parts) of listed
// tile k (lanes of one warp): a main tile by its geometry, a fix-up slot by
// its share of the fix-up list;
// owned says whether the tile's partial summed the cell (a main tile's
// cells of Coef.valid 1, a fix-up slot's of 3), so that no cell is taken
// twice.
template <typename F>
__device__ __forceinline__ void ref_tile_cells(const ScanArgs& A, int32_t j, int64_t k,
                                               int32_t part, int lane, F f) {
  if (k < A.n_tiles) {
    const TileGeom& g = A.geo;
    const int64_t tr = g.col_major ? k % g.ntr : k / g.ntc;
    const int64_t tc = g.col_major ? k / g.ntr : k % g.ntc;
    const int64_t r0 = tr * g.R, c0 = tc * g.C;
    const int64_t rows = min((int64_t)g.R, (int64_t)A.n_t0 - r0);
    const int64_t cols = min((int64_t)g.C, (int64_t)A.n_tau - c0);
    const int64_t n = rows * cols;
    for (int64_t q = n * part / A.parts + lane; q < n * (part + 1) / A.parts; q += 32) {
      const int64_t r = q / cols, cc = q - r * cols;
      const int64_t c = (r0 + r) * A.n_tau + c0 + cc;
      f(c, ref_valid_of(A.coef, A.shared, A.cells, j, c) == 1.0f);
    }
  } else {
    const int64_t cap = A.shared ? A.cells : A.cells * A.n_templates;
    const int64_t n = min((int64_t)*A.n_flag, cap);
    const int64_t b = k - A.n_tiles;
    int64_t lo, hi;
    fix_slot_range(b, n, kFixSlots, A.n_templates, &lo, &hi);
    const int64_t m = hi - lo;
    for (int64_t e = lo + m * part / A.parts + lane; e < lo + m * (part + 1) / A.parts; e += 32) {
      const int64_t entry = A.flag_list[e];
      if (!A.shared && entry / A.cells != j) continue;
      const int64_t c = A.shared ? entry : entry % A.cells;
      f(c, ref_valid_of(A.coef, A.shared, A.cells, j, c) == 3.0f);
    }
  }
}

// Passes 2 and 3 over the listed tiles' cells: the histogram (collect =
// false), which also keeps the cells in bins up to the tile pass's bound
// (cut[j]) while they fit kRefCandCap, then the cut and the collection of
// the cells up to it (collect = true): by the blocks (x, j) from the kept
// cells when they fit (the same set: every cell the cut takes lies in a bin
// <= cut[j]), else by a second scan of the tiles.  Grid (x, T), one warp per
// tile.  The histogram and the counts were cleared by the final reduction,
// the kept-cell count by the tile pass.
template <bool kCollect>
__global__ void __launch_bounds__(kRefThreads) k_ref_scan(const ScanArgs A) {
  __shared__ int32_t h[kRefBins];
  __shared__ int32_t s_last;
  const int32_t j = blockIdx.y;
  const int32_t n_kept = kCollect ? A.ref_ncand[j] : 0;
  const bool from_kept = kCollect && n_kept <= kRefCandCap;
  if (from_kept && (int64_t)blockIdx.x * kRefThreads >= n_kept) return;   // (past the list)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (kCollect) {
    for (int b = threadIdx.x; b < kRefBins; b += blockDim.x) h[b] = A.hist[(int64_t)j * kRefBins + b];
    __syncthreads();
    if (threadIdx.x == 0) s_last = ref_cut_of(h, A.cap, A.cut[j]);
  } else {
    for (int b = threadIdx.x; b < kRefBins; b += blockDim.x) h[b] = 0;
  }
  __syncthreads();
  const TStat s = A.st[j];
  const int32_t last = kCollect ? s_last : kRefBins - 1;
  const int32_t keep = kCollect ? -1 : A.cut[j];   // bins the histogram pass keeps
  if (from_kept) {   // the template's blocks share its kept list
    if (s.N <= 0 || last < 0) return;
    const float* mp = A.map + (int64_t)j * A.cells;
    const int32_t* cand = A.ref_cand + (int64_t)j * kRefCandCap;
    for (int32_t k = blockIdx.x * kRefThreads + threadIdx.x; k < n_kept;
         k += gridDim.x * kRefThreads) {
      const int32_t c = cand[k];
      const int b = ref_bin_of(mp[c], s.M);
      if (b >= 0 && b <= last) {
        const int32_t slot = atomicAdd(A.ref_n + j, 1);
        if (slot < kRefMaxCells) A.ref_cell[(int64_t)j * kRefMaxCells + slot] = c;
      }
    }
    return;
  }
  const int32_t nt = min(A.ref_ntile[j], kRefMaxTiles);
  if (s.N > 0 && last >= 0) {
    const float* mp = A.map + (int64_t)j * A.cells;
    const int64_t items = (int64_t)nt * A.parts;
    for (int64_t it = blockIdx.x * (kRefThreads / 32) + warp; it < items;
         it += gridDim.x * (kRefThreads / 32)) {
      const int64_t k = it / A.parts;
      ref_tile_cells(A, j, A.ref_tile[(int64_t)j * kRefMaxTiles + k], (int32_t)(it - k * A.parts),
                     lane, [&](int64_t c, bool owned) {
        int b = owned ? ref_bin_of(mp[c], s.M) : -1;
        if (b > last) b = -1;
        if (kCollect) {
          if (b >= 0) {
            const int32_t slot = atomicAdd(A.ref_n + j, 1);
            if (slot < kRefMaxCells) A.ref_cell[(int64_t)j * kRefMaxCells + slot] = (int32_t)c;
          }
        } else {
          // one shared-memory atomic per distinct bin among the lanes here
          // (noise maps put most cells of the window in a few bins)
          const unsigned act = __activemask();
          const unsigned peers = __match_any_sync(act, b);
          if (b >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h[b], __popc(peers));
          // keep the cells of bins <= keep: one global atomic per warp step
          const bool kept = b >= 0 && b <= keep;
          const unsigned sel = __ballot_sync(act, kept);
          if (sel) {
            const int leader = __ffs(sel) - 1;
            int32_t base = 0;
            if (lane == leader) base = atomicAdd(A.ref_ncand + j, __popc(sel));
            base = __shfl_sync(act, base, leader);
            const int32_t at = base + __popc(sel & ((1u << lane) - 1u));
            if (kept && at < kRefCandCap) A.ref_cand[(int64_t)j * kRefCandCap + at] = (int32_t)c;
          }
        }
      });
    }
  }
  if (!kCollect) {
    __syncthreads();
    for (int b = threadIdx.x; b < kRefBins; b += blockDim.x)
      if (h[b]) atomicAdd(A.hist + (int64_t)j * kRefBins + b, h[b]);
  }
}

struct RefArgs {
  const int32_t* rel_t;
  const int64_t* t_base;
  int32_t n_sft;
  fmap_grid g;
  const int64_t* ax;
  const float2* wtab;
  int32_t n_tab;
  const int32_t* i0;
  const int32_t* jend;
  const float* antenna;
  const float* fafb;
  int32_t shared;
  float* map;
  int64_t cells;
  const int32_t* ref_n;
  const int32_t* ref_cell;
  float* ref_fast;
  double* ref_val;
};

// Pass 3: one warp per collected cell.  The lanes split the window's atoms
// into 32 contiguous runs and sum them in float-float arithmetic (a value is
// an unevaluated pair h + l, ~2^-44 relative; GB300 runs FP64 at 1/64 of the
// FP32 rate): an exponential run takes its first weight from an FP64 exp and
// the rest as products of per-gap decays (e^{-T_sft/tau} for one-SFT gaps), a
// table window evaluates w per atom in FP64, a rectangular one has w = 1.  The
// seven sums meet in a fixed butterfly; lane 0 forms D and 2F in FP64 from
// them, records the fast and refined values and writes the refined value to
// the map.

__device__ __forceinline__ void ref_cell_one(const RefArgs& A, int32_t j, int32_t k, int lane) {
  const fmap_grid& g = A.g;
  const int64_t slot = (int64_t)j * kRefMaxCells + k;
  const int32_t c = A.ref_cell[slot];
  const int32_t m = c / g.n_tau, nn = c - m * g.n_tau;
  const int32_t i0 = A.i0[m], je = A.jend[c];
  const int32_t len = max(0, je - i0);
  const int64_t t0rel = grid_t0(g, A.ax, m) - *A.t_base;
  const int64_t tau = grid_tau(g, A.ax, nn);
  const double inv_tau = 1.0 / (double)tau;
  const int32_t a_lo = i0 + (int32_t)((int64_t)len * lane / 32);
  const int32_t a_hi = i0 + (int32_t)((int64_t)len * (lane + 1) / 32);
  const int64_t n = A.n_sft;
  const float* ant = A.antenna + (A.shared ? 0 : (int64_t)j * 3 * n);
  const float* x = A.fafb + (int64_t)j * 4 * n;
  const bool ex = g.window == FMAP_EXP, tw = g.window == FMAP_TABLE;
  const double su = tw ? tab_scale(A.n_tab, exp_cut8_of(g), tau) : 0.0;
  FF s[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) s[q] = FF{0.0f, 0.0f};
  if (a_lo < a_hi) {
    FF w{1.0f, 0.0f}, rho1{1.0f, 0.0f};
    if (ex) {
      w = ff_of(exp(-(double)((int64_t)A.rel_t[a_lo] - t0rel) * inv_tau));
      rho1 = ff_of(exp(-(double)g.t_sft * inv_tau));
    }
    for (int32_t a = a_lo; a < a_hi; ++a) {
      if (ex && a > a_lo) {
        const int32_t gap = A.rel_t[a] - A.rel_t[a - 1];
        w = ff_mul(w, gap == (int32_t)g.t_sft ? rho1 : ff_of(exp(-(double)gap * inv_tau)));
      }
      if (tw) w = ff_of(tab_weight64((double)((int64_t)A.rel_t[a] - t0rel) * su, A.wtab, A.n_tab));
      if (g.window == FMAP_RECT) {
        s[0] = ff_add(s[0], FF{ant[a], 0.0f});
        s[1] = ff_add(s[1], FF{ant[n + a], 0.0f});
        s[2] = ff_add(s[2], FF{ant[2 * n + a], 0.0f});
        s[3] = ff_add(s[3], FF{x[a], 0.0f});
        s[4] = ff_add(s[4], FF{x[n + a], 0.0f});
        s[5] = ff_add(s[5], FF{x[2 * n + a], 0.0f});
        s[6] = ff_add(s[6], FF{x[3 * n + a], 0.0f});
      } else {
        const FF w2 = ff_mul(w, w);
        ff_acc(s[0], w2, ant[a]);
        ff_acc(s[1], w2, ant[n + a]);
        ff_acc(s[2], w2, ant[2 * n + a]);
        ff_acc(s[3], w, x[a]);
        ff_acc(s[4], w, x[n + a]);
        ff_acc(s[5], w, x[2 * n + a]);
        ff_acc(s[6], w, x[3 * n + a]);
      }
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1)
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const FF o{__shfl_xor_sync(0xffffffffu, s[q].h, d), __shfl_xor_sync(0xffffffffu, s[q].l, d)};
      s[q] = ff_add(s[q], o);
    }
  if (lane == 0) {
    double v7[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) v7[q] = (double)s[q].h + (double)s[q].l;
    const double Aa = v7[0], Bb = v7[1], Cc = v7[2];
    const double D = Aa * Bb - Cc * Cc;
    const bool ok = len >= 2 && D > 0.0;
    double v = 0.0;
    if (ok)
      v = 2.0 * (Bb * (v7[3] * v7[3] + v7[4] * v7[4]) + Aa * (v7[5] * v7[5] + v7[6] * v7[6]) -
                 2.0 * Cc * (v7[3] * v7[5] + v7[4] * v7[6])) / D;
    float* mp = A.map + (int64_t)j * A.cells + c;
    A.ref_fast[slot] = *mp;
    A.ref_val[slot] = ok ? v : -1.0;
    *mp = (float)v;
  }
}

__global__ void __launch_bounds__(kRefThreads) k_ref_cells(const RefArgs A) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t j = blockIdx.y;
  const int32_t n_cand = min(A.ref_n[j], kRefMaxCells);
  for (int32_t k = blockIdx.x * (kRefThreads / 32) + warp; k < n_cand;
       k += gridDim.x * (kRefThreads / 32))
    ref_cell_one(A, j, k, lane);
}

// Pass 4: one block per template rebuilds its summary from the fast
// statistics and the collected cells.  Every exp-term is in (0, 1] (relative
// to the fast or the refined maximum, both held by a collected cell) and is
// summed as an integer in 2^-51 units, so the sums do not depend on the
// order in which the cells were collected (<= 4096 terms <= 2^63: no overflow,
// relative error < 1e-12).
constexpr int kFinalThreads = 256;

__global__ void __launch_bounds__(kFinalThreads)
k_ref_final(const TStat* __restrict__ st, const int32_t* __restrict__ hist,
            const int32_t* __restrict__ cut, int32_t cap, const int32_t* __restrict__ ref_ntile,
            const int32_t* __restrict__ ref_n, const int32_t* __restrict__ ref_cell,
            const float* __restrict__ ref_fast, const double* __restrict__ ref_val, int32_t n_tau,
            double log_prior, double tol, fmap_summary* __restrict__ out) {
  constexpr int NW = kFinalThreads / 32;
  __shared__ double s_mx[NW];
  __shared__ unsigned long long s_sub[NW], s_add[NW];
  __shared__ long long s_nv[NW];
  __shared__ int32_t s_arg[NW];
  const int32_t j = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TStat s = st[j];
  const int32_t n = min(ref_n[j], kRefMaxCells);
  if (s.N <= 0 || n <= 0) return;   // the fast summary stands (flags 0)
  const int64_t base = (int64_t)j * kRefMaxCells;
  double mx = -1.0;
  for (int32_t k = threadIdx.x; k < n; k += kFinalThreads) mx = fmax(mx, ref_val[base + k]);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, d));
  if (lane == 0) s_mx[warp] = mx;
  __syncthreads();
#pragma unroll
  for (int w = 0; w < NW; ++w) mx = fmax(mx, s_mx[w]);
  if (mx < 0.0) return;   // no collected cell valid in FP64: keep the fast summary
  constexpr double kFix = 2251799813685248.0;   // 2^51
  unsigned long long sub = 0ull, add = 0ull;
  long long nv = 0;
  int32_t arg = 0x7fffffff;
  const double M = (double)s.M;
  for (int32_t k = threadIdx.x; k < n; k += kFinalThreads) {
    const double ef = exp(0.5 * fmin((double)ref_fast[base + k] - M, 0.0));
    sub += (unsigned long long)__double2ull_rn(ef * kFix);
    const double v = ref_val[base + k];
    if (v >= 0.0) {
      add += (unsigned long long)__double2ull_rn(exp(0.5 * (v - mx)) * kFix);
      nv += 1;
      if (v == mx) arg = min(arg, ref_cell[base + k]);
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    sub += __shfl_xor_sync(0xffffffffu, sub, d);
    add += __shfl_xor_sync(0xffffffffu, add, d);
    nv += __shfl_xor_sync(0xffffffffu, nv, d);
    arg = min(arg, __shfl_xor_sync(0xffffffffu, arg, d));
  }
  if (lane == 0) {
    s_sub[warp] = sub;
    s_add[warp] = add;
    s_nv[warp] = nv;
    s_arg[warp] = arg;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < NW; ++w) {   // (integer sums: the order does not matter)
    sub += s_sub[w];
    add += s_add[w];
    nv += s_nv[w];
    arg = min(arg, s_arg[w]);
  }
  const double Sp = exp(0.5 * (M - mx)) * fmax(s.S - (double)sub / kFix, 0.0) + (double)add / kFix;
  const long long Np = s.N - n + nv;
  const int32_t b = ref_cut_of(hist + (int64_t)j * kRefBins, cap, cut[j]);
  const double depth = b + 1 >= kRefBins ? (double)kRefWindow
                                         : (double)(b + 1) * (double)kRefWindow / kRefBins;
  fmap_summary o;
  o.max2F = (float)mx;
  o.m = arg / n_tau;
  o.n = arg % n_tau;
  const bool complete = ref_ntile[j] <= kRefMaxTiles;   // every candidate tile scanned
  o.flags = (int32_t)FMAP_SUMMARY_REFINED |
            (complete && depth > 2.0 * tol * fmax(mx, 1.0) ? (int32_t)FMAP_SUMMARY_ARGMAX_EXACT
                                                            : 0);
  o.logB = 0.5 * mx + log(Sp) - log((double)Np) + log_prior;
  o.n_valid = Np;
  out[j] = o;
}

cudaError_t launch_refine(fmap_plan_s* p, const fmap_atoms* a, float* d_2F,
                          fmap_summary* d_summary, int64_t n_tiles, cudaStream_t s) {
  const int32_t cap = refine_cells_of(p);
  const fmap_grid& g = p->grid;
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const int32_t T = p->n_templates;
  if (cap <= 0 || !d_2F || !d_summary || T == 0 || cells == 0 || p->n_sft == 0)
    return cudaSuccess;
  Workspace& w = p->ws;
  const int32_t sh = a->shared_antenna ? 1 : 0;
  // (the final reduction cleared the cell histogram and the candidate counts)
  k_ref_tiles<<<T, kTileThreads, 0, s>>>(w.partials, p->part_stride, n_tiles, p->n_tiles, kFixSlots,
                                        w.tstat, cap, w.ref_ntile, w.ref_tile, w.ref_bin,
                                        w.ref_ncand);
  ScanArgs S;
  S.map = d_2F;
  S.coef = w.coef;
  S.shared = sh;
  S.n_t0 = g.n_t0;
  S.n_tau = g.n_tau;
  S.cells = cells;
  S.geo = p->tiles;
  S.n_tiles = n_tiles;
  S.flag_list = w.flag_list;
  S.n_flag = w.n_flag;
  S.n_templates = T;
  S.st = w.tstat;
  S.ref_ntile = w.ref_ntile;
  S.ref_tile = w.ref_tile;
  S.hist = w.ref_hist;
  S.cap = cap;
  S.cut = w.ref_bin;
  S.ref_n = w.ref_n;
  S.ref_cell = w.ref_cell;
  S.ref_ncand = w.ref_ncand;
  S.ref_cand = w.ref_cand;
  // a warp per share of about kScanShare cells of a listed tile (about cap
  // tiles per template), at least a few blocks over the GPU
  const int64_t tile_cells = (int64_t)S.geo.R * S.geo.C;
  S.parts = (int32_t)std::min<int64_t>(std::max<int64_t>((tile_cells + kScanShare - 1) / kScanShare, 1),
                                       1024);
  const int wpb = kRefThreads / 32;
  const unsigned gx = (unsigned)std::max<int64_t>(
      (2 * (int64_t)cap * S.parts + wpb - 1) / wpb, ((int64_t)p->n_sm * 4 + T - 1) / T);
  const dim3 grid(std::min<unsigned>(gx, 4096u), (unsigned)T);
  k_ref_scan<false><<<grid, kRefThreads, 0, s>>>(S);
  k_ref_scan<true><<<grid, kRefThreads, 0, s>>>(S);
  RefArgs A;
  A.rel_t = w.rel_t;
  A.t_base = w.t_base;
  A.n_sft = p->n_sft;
  A.g = g;
  A.ax = plan_axes(p);
  A.wtab = w.wtab;
  A.n_tab = p->n_tab;
  A.i0 = w.i0;
  A.jend = w.jend;
  A.antenna = a->antenna;
  A.fafb = a->fafb;
  A.shared = sh;
  A.map = d_2F;
  A.cells = cells;
  A.ref_n = w.ref_n;
  A.ref_cell = w.ref_cell;
  A.ref_fast = w.ref_fast;
  A.ref_val = w.ref_val;
  k_ref_cells<<<dim3((unsigned)((cap + wpb - 1) / wpb), (unsigned)T), kRefThreads, 0, s>>>(A);
  k_ref_final<<<T, kFinalThreads, 0, s>>>(w.tstat, w.ref_hist, w.ref_bin, cap, w.ref_ntile, w.ref_n,
                               w.ref_cell, w.ref_fast, w.ref_val, g.n_tau, p->log_prior,
                               fast_tol(p), d_summary);
  p->launches += 5;
  return cudaGetLastError();
}

}  // namespace fmap
