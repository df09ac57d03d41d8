// Kernels shared by both windows: input preparation, the window index tables
// (Eq. Fmn grid, window membership of Eq. winrect / winexp), the final
// per-template reduction and the standalone marginalisation.
#include <math.h>

#include "fmap_batch.cuh"
#include "fmap_device.cuh"

namespace fmap {

// Non-finite check of n values (antenna or data rows): DEV_ERR_NONFINITE
// is latched if any is NaN or infinite (|x| <= FLT_MAX fails for both; one
// atomic per warp at most).
__device__ __forceinline__ void finite_check(const float* __restrict__ v, int64_t n,
                                             int64_t i0, int64_t step, uint32_t* __restrict__ err) {
  bool bad = false;
  for (int64_t i = i0; i < n; i += step) bad |= !(fabsf(v[i]) <= 3.402823466e38f);
  const unsigned who = __ballot_sync(__activemask(), bad);
  if (bad && (int)(threadIdx.x & 31) == __ffs(who) - 1) atomicOr(err, DEV_ERR_NONFINITE);
}

// t -> t - t[0] as int32, with the data checks (strictly increasing,
// span < 2^31 s) latched into the plan's status word, and the atoms' values
// checked for NaN and infinities.
__device__ __forceinline__ void prep_body(const int64_t* __restrict__ t, int32_t n, int32_t n_alloc,
                       int32_t* __restrict__ rel_t, int64_t* __restrict__ t_base,
                       uint32_t* __restrict__ err, const float* __restrict__ ant, int64_t n_ant_vals,
                       const float* __restrict__ x, int64_t n_x_vals,
    const uint3 bid, const dim3 gdim) {
  {
    const int64_t g0 = bid.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t step = (int64_t)gdim.x * blockDim.x;
    if (ant) finite_check(ant, n_ant_vals, g0, step, err);
    if (x) finite_check(x, n_x_vals, g0, step, err);
  }
  if (n <= 0) return;
  const int64_t base = t[0];
  for (int64_t i = n + bid.x * (int64_t)blockDim.x + threadIdx.x; i < n_alloc;
       i += (int64_t)gdim.x * blockDim.x)
    rel_t[i] = 0;
  for (int64_t i = bid.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gdim.x * blockDim.x) {
    const int64_t ti = t[i];
    const int64_t d = ti - base;
    uint32_t e = 0;
    if (d < 0 || d > 0x7fffffffLL - 1) e |= DEV_ERR_SPAN;
    if (i + 1 < n && t[i + 1] <= ti) e |= DEV_ERR_ORDER;
    if (e) atomicOr(err, e);
    rel_t[i] = (int32_t)(d & 0x7fffffffLL);
    if (i == 0) *t_base = base;
  }
}

__global__ void k_prep(const int64_t* __restrict__ t, int32_t n, int32_t n_alloc,
                       int32_t* __restrict__ rel_t, int64_t* __restrict__ t_base,
                       uint32_t* __restrict__ err, const float* __restrict__ ant,
                       int64_t n_ant_vals, const float* __restrict__ x, int64_t n_x_vals) {
  prep_body(t, n, n_alloc, rel_t, t_base, err, ant, n_ant_vals, x, n_x_vals, blockIdx, gridDim);
}

// Window index tables: i0[m] = first atom with t >= t0_m; jend[m][n] = one
// past the last atom whose SFT ends by t0_m + L_n (L = window_len(tau_n)),
// clamped to >= i0[m], so the window holds atoms [i0, jend).  One block per
// group of kIdxGroup t0 rows: each warp finds one row's atom range
// [i0, j(n_tau - 1)) by a warp-wide search, the union of the group's ranges
// of relative times is staged in shared memory once (coalesced), and every
// (row, tau) searches it there; longer unions search global memory.
constexpr int kIdxThreads = 256;
constexpr int kIdxGroup = kIdxThreads / 32;   // t0 rows per block pass (one warp each)
constexpr int kIdxCap = 8192;   // staged relative times (32 KB)

// First index in [lo, hi) of the ascending int32 times with t > x (int64).
__device__ __forceinline__ int32_t upper_bound_i32(const int32_t* t, int32_t lo, int32_t hi,
                                                   int64_t x) {
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if ((int64_t)t[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// The same search by one whole warp: 32 probes per round narrow the range
// 32-fold, so a data set of N atoms takes ~log32(N) dependent loads instead
// of log2(N).  Returns the first index in [lo, hi) whose time exceeds x (hi
// if none) to every lane.
__device__ __forceinline__ int32_t warp_upper_bound_i32(const int32_t* t, int32_t lo, int32_t hi,
                                                        int64_t x, int lane) {
  while (hi - lo > 32) {
    const int32_t step = (hi - lo + 31) / 32;
    const int32_t p = lo + lane * step;
    const bool le = p < hi && (int64_t)t[p] <= x;   // the probes below the answer
    const int c = __popc(__ballot_sync(0xffffffffu, le));
    if (c == 0) return lo;
    const int32_t base = lo;
    lo = base + (c - 1) * step + 1;
    hi = min(hi, base + c * step);
  }
  const int32_t p = lo + lane;
  const bool le = p < hi && (int64_t)t[p] <= x;
  return lo + __popc(__ballot_sync(0xffffffffu, le));
}

__device__ __forceinline__ void index_body(const int32_t* __restrict__ rel_t,
                                           const int64_t* __restrict__ t_base, int32_t n_sft,
                                           fmap_grid g, const int64_t* __restrict__ ax,
                                           int32_t* __restrict__ i0tab,
                                           int32_t* __restrict__ jend, int32_t m0, int32_t R) {
  __shared__ int32_t s_t[kIdxCap];
  __shared__ int32_t s_lo[kIdxGroup], s_hi[kIdxGroup];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t tb = n_sft > 0 ? *t_base : 0;
  const int64_t lmax = window_len(g, grid_tau(g, ax, g.n_tau - 1)) - g.t_sft;
  if (warp < R) {   // warp r: row m0 + r's first atom with t >= t0 and the last any window takes
    const int32_t m = m0 + warp;
    const int64_t t0rel = grid_t0(g, ax, m) - tb;
    const int32_t lo = warp_upper_bound_i32(rel_t, 0, n_sft, t0rel - 1, lane);
    const int32_t hi = max(lo, warp_upper_bound_i32(rel_t, lo, n_sft, t0rel + lmax, lane));
    if (lane == 0) {
      s_lo[warp] = lo;
      s_hi[warp] = hi;
      i0tab[m] = lo;
    }
  }
  __syncthreads();
  // Both ends grow with t0, so the group's rows search within [lo of its
  // first row, hi of its last), staged once when it fits.
  const int32_t base = s_lo[0], span = s_hi[R - 1] - base;
  const bool staged = span <= kIdxCap;
  if (staged)
    for (int k = tid; k < span; k += kIdxThreads) s_t[k] = rel_t[base + k];
  __syncthreads();
  for (int32_t r = 0; r < R; ++r) {   // no barrier between rows: their searches overlap
    const int32_t m = m0 + r, lo = s_lo[r], hi = s_hi[r];
    const int64_t t0rel = grid_t0(g, ax, m) - tb;
    int32_t* row = jend + (int64_t)m * g.n_tau;
    for (int32_t nn = tid; nn < g.n_tau; nn += kIdxThreads) {
      const int64_t lim = t0rel + window_len(g, grid_tau(g, ax, nn)) - g.t_sft;
      row[nn] = staged ? base + upper_bound_i32(s_t, lo - base, hi - base, lim)
                       : upper_bound_i32(rel_t, lo, hi, lim);
    }
  }
  __syncthreads();   // s_t, s_lo and s_hi are reused by the block's next group
}

__global__ void __launch_bounds__(kIdxThreads)
k_index(const int32_t* __restrict__ rel_t, const int64_t* __restrict__ t_base, int32_t n_sft,
        fmap_grid g, const int64_t* __restrict__ ax, int32_t* __restrict__ i0tab,
        int32_t* __restrict__ jend, int32_t grp) {
  const int32_t n_grp = (g.n_t0 + grp - 1) / grp;
  for (int32_t q = blockIdx.x; q < n_grp; q += gridDim.x)
    index_body(rel_t, t_base, n_sft, g, ax, i0tab, jend, q * grp, min(grp, g.n_t0 - q * grp));
}

cudaError_t launch_prep(fmap_plan_s* p, const fmap_atoms* a, cudaStream_t s) {
  if (p->n_sft <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t n = p->n_sft;
  const int64_t n_ant = 3 * n * (a->shared_antenna ? 1 : std::max<int32_t>(p->n_templates, 1));
  const int64_t n_x = 4 * n * (int64_t)p->n_templates;
  // enough threads for the timestamps, and for the value checks at a few
  // values per thread
  const int64_t want = std::max<int64_t>(n, (n_ant + n_x) / 8);
  const int blocks = (int)std::min<int64_t>((want + threads - 1) / threads, (int64_t)p->n_sm * 16);
  k_prep<<<std::max(blocks, 1), threads, 0, s>>>(a->t, p->n_sft, rel_t_entries(p->n_sft),
                                                 p->ws.rel_t, p->ws.t_base, p->ws.dev_err,
                                                 a->antenna, n_ant, a->fafb, n_x);
  p->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_index(fmap_plan_s* p, const int64_t* d_t, cudaStream_t s) {
  (void)d_t;
  const int64_t cells = (int64_t)p->grid.n_t0 * p->grid.n_tau;
  if (cells == 0) return cudaSuccess;
  // rows per group: as many as keep about four blocks per SM busy (1..8)
  const int32_t grp = (int32_t)std::max<int64_t>(
      1, std::min<int64_t>(kIdxGroup, p->grid.n_t0 / ((int64_t)p->n_sm * 4)));
  const int blocks = (int)std::min<int64_t>((p->grid.n_t0 + grp - 1) / grp, (int64_t)p->n_sm * 8);
  k_index<<<blocks, kIdxThreads, 0, s>>>(p->ws.rel_t, p->ws.t_base, p->n_sft, p->grid, plan_axes(p),
                                         p->ws.i0, p->ws.jend, grp);
  p->launches += 1;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Final reduction in two levels, accumulated in FP64: level 1 merges groups of
// kRedGroup tile partials per template (many blocks), level 2 merges the
// groups of one template (one block).  Each level fixes the order of its
// additions (per-thread strided loop, then a fixed tree), so the result is
// deterministic.
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedGroup = 2048;

struct __align__(32) Partial64 {
  double sum;      // sum of exp(F - max2F/2) over the group's valid cells
  float max2F;
  int32_t arg;
  long long nvalid;
  long long pad;
};

// Block-wide (max, count) then (sum, min arg at max) over items get(b),
// b in [0, n).  Returns the block's merged partial in thread 0.
template <typename Get>
__device__ __forceinline__ Partial64 block_merge(int64_t n, Get get) {
  __shared__ float s_max[kRedThreads];
  __shared__ long long s_cnt[kRedThreads];
  __shared__ double s_sum[kRedThreads];
  __shared__ int32_t s_arg[kRedThreads];
  const int tid = threadIdx.x;
  float mx = -1.0f;
  long long cnt = 0;
  for (int64_t b = tid; b < n; b += kRedThreads) {
    const Partial64 q = get(b);
    if (q.nvalid > 0) {
      mx = fmaxf(mx, q.max2F);
      cnt += q.nvalid;
    }
  }
  s_max[tid] = mx;
  s_cnt[tid] = cnt;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (tid < w) {
      s_max[tid] = fmaxf(s_max[tid], s_max[tid + w]);
      s_cnt[tid] += s_cnt[tid + w];
    }
    __syncthreads();
  }
  const float M = s_max[0];
  const long long N = s_cnt[0];
  __syncthreads();
  double sum = 0.0;
  int32_t arg = kNoArg;
  if (N > 0) {
    for (int64_t b = tid; b < n; b += kRedThreads) {
      const Partial64 q = get(b);
      if (q.nvalid > 0) {
        // Rescale factor exp((max2F - M) / 2) <= 1 in FP32 (relative error
        // ~1e-7, the order of the FP32 tile sums themselves), accumulated in
        // FP64; factors below 2^-126 flush to 0.
        float f;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"((q.max2F - M) * 0.72134752044448170368f));
        sum += q.sum * (double)f;
        if (q.max2F == M && q.arg < arg) arg = q.arg;
      }
    }
  }
  s_sum[tid] = sum;
  s_arg[tid] = arg;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (tid < w) {
      s_sum[tid] += s_sum[tid + w];
      s_arg[tid] = min(s_arg[tid], s_arg[tid + w]);
    }
    __syncthreads();
  }
  Partial64 r;
  r.sum = s_sum[0];
  r.max2F = M;
  r.arg = s_arg[0];
  r.nvalid = N;
  r.pad = 0;
  return r;
}

__device__ __forceinline__ Partial64 widen(const Partial& q) {
  Partial64 r;
  r.sum = (double)q.sum;
  r.max2F = q.max2F;
  r.arg = q.arg;
  r.nvalid = q.nvalid;
  r.pad = 0;
  return r;
}

// Level 1: block (g, t) merges slots [g*kRedGroup, (g+1)*kRedGroup) of the
// concatenation [main tiles 0..n_tiles) ++ [fix-up slots fix0..fix0+n_fix).
__device__ __forceinline__ void reduce_groups_body(const Partial* __restrict__ parts, int64_t n_tiles, int64_t fix0, int64_t n_fix,
                int64_t stride, int64_t n_groups, Partial64* __restrict__ groups,
    const uint3 bid, const dim3 gdim) {
  const Partial* pp = parts + (int64_t)bid.y * stride;
  const int64_t n_all = n_tiles + n_fix;
  const int64_t lo = (int64_t)bid.x * kRedGroup;
  const int64_t n = max((int64_t)0, min((int64_t)kRedGroup, n_all - lo));
  const Partial64 r = block_merge(n, [&](int64_t b) {
    const int64_t k = lo + b;
    return widen(k < n_tiles ? pp[k] : pp[fix0 + (k - n_tiles)]);
  });
  if (threadIdx.x == 0) groups[(int64_t)bid.y * n_groups + bid.x] = r;
}

__global__ void __launch_bounds__(kRedThreads)
k_reduce_groups(const Partial* __restrict__ parts, int64_t n_tiles, int64_t fix0, int64_t n_fix,
                int64_t stride, int64_t n_groups, Partial64* __restrict__ groups) {
  reduce_groups_body(parts, n_tiles, fix0, n_fix, stride, n_groups, groups, blockIdx, gridDim);
}

// Level 2: one block per template over its groups; writes the summary and,
// when tstat is given, the statistics the refinement starts from (and clears
// that template's refinement histogram and candidate count).
__device__ __forceinline__ void reduce_final_body(const Partial64* __restrict__ groups, int64_t n_groups, int32_t n_tau,
               double log_prior, fmap_summary* __restrict__ out, TStat* __restrict__ tstat,
    const uint3 bid, const dim3 gdim, int32_t* __restrict__ ref_hist = nullptr,
    int32_t* __restrict__ ref_n = nullptr) {
  if (ref_hist) {
    for (int b = threadIdx.x; b < kRefBins; b += blockDim.x) ref_hist[(int64_t)bid.x * kRefBins + b] = 0;
    if (threadIdx.x == 0) ref_n[bid.x] = 0;
  }
  const Partial64* gp = groups + (int64_t)bid.x * n_groups;
  const Partial64 r = block_merge(n_groups, [&](int64_t b) { return gp[b]; });
  if (threadIdx.x == 0) {
    if (tstat) {
      TStat t;
      t.S = r.sum;
      t.M = r.max2F;
      t.arg = r.arg;
      t.N = r.nvalid;
      t.pad = 0;
      tstat[bid.x] = t;
    }
    fmap_summary o;
    o.flags = 0;
    o.n_valid = r.nvalid;
    if (r.nvalid == 0) {
      o.max2F = 0.0f;
      o.m = -1;
      o.n = -1;
      o.logB = nan("");
    } else {
      o.max2F = r.max2F;
      o.m = r.arg / n_tau;
      o.n = r.arg % n_tau;
      o.logB = 0.5 * (double)r.max2F + log(r.sum) - log((double)r.nvalid) + log_prior;
    }
    out[bid.x] = o;
  }
}

__global__ void __launch_bounds__(kRedThreads)
k_reduce_final(const Partial64* __restrict__ groups, int64_t n_groups, int32_t n_tau,
               double log_prior, fmap_summary* __restrict__ out, TStat* __restrict__ tstat,
               int32_t* __restrict__ ref_hist, int32_t* __restrict__ ref_n) {
  reduce_final_body(groups, n_groups, n_tau, log_prior, out, tstat, blockIdx, gridDim, ref_hist,
                    ref_n);
}

int64_t reduce_groups_of(int64_t slots) { return std::max<int64_t>(1, (slots + kRedGroup - 1) / kRedGroup); }

static cudaError_t reduce_into(const Partial* parts, int64_t n_tiles, int64_t fix0, int64_t n_fix,
                               int64_t stride, int32_t T, int32_t n_tau, double log_prior,
                               Partial64* groups, fmap_summary* d_summary, cudaStream_t s,
                               TStat* tstat = nullptr, int32_t* ref_hist = nullptr,
                               int32_t* ref_n = nullptr) {
  const int64_t n_groups = reduce_groups_of(n_tiles + n_fix);
  k_reduce_groups<<<dim3((unsigned)n_groups, (unsigned)T), kRedThreads, 0, s>>>(
      parts, n_tiles, fix0, n_fix, stride, n_groups, groups);
  k_reduce_final<<<T, kRedThreads, 0, s>>>(groups, n_groups, n_tau > 0 ? n_tau : 1, log_prior,
                                           d_summary, tstat, ref_hist, ref_n);
  return cudaGetLastError();
}

cudaError_t launch_final_reduce(fmap_plan_s* p, int64_t n_tiles, bool with_fix,
                                fmap_summary* d_summary, cudaStream_t s) {
  if (!d_summary || p->n_templates == 0) return cudaSuccess;
  const bool fix = with_fix && (int64_t)p->grid.n_t0 * p->grid.n_tau > 0;
  p->launches += 2;
  return reduce_into(p->ws.partials, n_tiles, p->n_tiles, fix ? kFixSlots : 0, p->part_stride,
                     p->n_templates, p->grid.n_tau, p->log_prior, (Partial64*)p->ws.groups,
                     d_summary, s, p->ws.tstat, p->ws.ref_hist, p->ws.ref_n);
}

// ---------------------------------------------------------------------------
// Standalone marginalisation of a given map: 2048 cells per tile.
// ---------------------------------------------------------------------------
constexpr int kMargThreads = 256;
constexpr int kMargPer = 8;

int64_t marg_tiles(const fmap_grid& g) {
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  return (cells + kMargThreads * kMargPer - 1) / (kMargThreads * kMargPer);
}

__global__ void __launch_bounds__(kMargThreads)
k_marg_partials(const float* __restrict__ map, const uint8_t* __restrict__ valid, int64_t cells,
                int64_t stride, Partial* __restrict__ parts) {
  __shared__ Partial scratch[kMargThreads / 32];
  const int64_t tile = blockIdx.x;
  const int64_t tmpl = blockIdx.y;
  const float* mp = map + tmpl * cells;
  const uint8_t* vp = valid ? valid + tmpl * cells : nullptr;
  Partial acc = partial_empty();
  const int64_t base = tile * (kMargThreads * kMargPer);
#pragma unroll
  for (int k = 0; k < kMargPer; ++k) {
    const int64_t c = base + k * kMargThreads + threadIdx.x;
    if (c < cells) {
      const bool ok = vp ? (vp[c] != 0) : true;
      partial_add(acc, mp[c], (int32_t)c, ok);
    }
  }
  acc = partial_block_reduce<kMargThreads / 32>(acc, scratch);
  if (threadIdx.x == 0) parts[tmpl * stride + tile] = acc;
}

cudaError_t launch_marginalise_into(const fmap_grid& g, int32_t n_templates, const float* d_2F,
                                    const uint8_t* d_valid, Partial* parts, double log_prior,
                                    fmap_summary* d_summary, cudaStream_t s) {
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const int64_t tiles = marg_tiles(g);
  if (n_templates == 0) return cudaSuccess;
  if (tiles > 0) {
    dim3 grid((unsigned)tiles, (unsigned)n_templates);
    k_marg_partials<<<grid, kMargThreads, 0, s>>>(d_2F, d_valid, cells, tiles, parts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // the group results of the first level follow the tile partials
  Partial64* groups = (Partial64*)(parts + (int64_t)n_templates * tiles);
  groups = (Partial64*)(((uintptr_t)groups + 31) & ~(uintptr_t)31);
  return reduce_into(parts, tiles, 0, 0, tiles, n_templates, g.n_tau, log_prior, groups,
                     d_summary, s);
}

cudaError_t launch_marginalise(fmap_plan_s* p, const float* d_2F, const uint8_t* d_valid,
                               fmap_summary* d_summary, cudaStream_t s) {
  const int64_t cells = (int64_t)p->grid.n_t0 * p->grid.n_tau;
  const int64_t tiles = marg_tiles(p->grid);
  if (tiles > 0 && p->n_templates > 0) {
    dim3 grid((unsigned)tiles, (unsigned)p->n_templates);
    k_marg_partials<<<grid, kMargThreads, 0, s>>>(d_2F, d_valid, cells, p->part_stride,
                                                  p->ws.partials);
    p->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_final_reduce(p, tiles, false, d_summary, s);
}


// ---- persistent multi-instance dispatchers (uneven batches) ----
__global__ void __launch_bounds__(256) kb_prep(const BItem* __restrict__ items, BUnits u) {
  // units [0, ru): relative times; then the marked-entry bitmask is cleared
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    const int64_t ru = it.n_sft > 0 ? (it.n_alloc + 255) / 256 : 0;
    if (k < ru) {
      prep_body(it.t, it.n_sft, it.n_alloc, it.rel_t, it.t_base, it.dev_err, it.antenna,
                (int64_t)3 * it.n_sft * it.n_ant, it.fafb, (int64_t)4 * it.n_sft * it.T,
                make_uint3((unsigned)k, 0, 0), dim3((unsigned)ru));
    } else {
      const int64_t w0 = (k - ru) * kBitsPerUnit;
      const int64_t w1 = min(flag_words(it.flag_entries), w0 + kBitsPerUnit);
      for (int64_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) it.flag_bits[w] = 0u;
    }
  });
}
static_assert(kIdxRowsPerUnit == kIdxGroup, "a batch index unit is one row group");
__global__ void __launch_bounds__(kIdxThreads) kb_index(const BItem* __restrict__ items, BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    const int32_t m0 = (int32_t)k * kIdxRowsPerUnit;
    index_body(it.rel_t, it.t_base, it.n_sft, it.g, it.ax, it.i0, it.jend, m0,
               min(kIdxRowsPerUnit, it.g.n_t0 - m0));
  });
}
__global__ void __launch_bounds__(kRedThreads) kb_red_groups(const BItem* __restrict__ items,
                                                             BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    const int64_t fix = it.cells > 0 ? kFixSlots : 0;
    reduce_groups_body(it.partials, it.tiles_used, it.n_tiles, fix, it.part_stride, it.red_groups,
                       (Partial64*)it.red_buf,
                       make_uint3((unsigned)(k % it.red_groups), (unsigned)(k / it.red_groups), 0),
                       dim3((unsigned)it.red_groups, (unsigned)it.T));
  });
}
__global__ void __launch_bounds__(kRedThreads) kb_red_final(const BItem* __restrict__ items,
                                                            BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    reduce_final_body((const Partial64*)it.red_buf, it.red_groups, it.g.n_tau > 0 ? it.g.n_tau : 1,
                      it.log_prior, it.summary, nullptr, make_uint3((unsigned)k, 0, 0),
                      dim3((unsigned)it.T));
  });
}
const void* batch_kernel_common(int phase) {
  switch (phase) {
    case BP_PREP: return (const void*)kb_prep;
    case BP_INDEX: return (const void*)kb_index;
    case BP_RED_GROUPS: return (const void*)kb_red_groups;
    case BP_RED_FINAL: return (const void*)kb_red_final;
  }
  return nullptr;
}

}  // namespace fmap
