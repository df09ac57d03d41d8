// Ill-conditioned cells.
//
// 2F depends on the component of (Fa, Fb) along the weak eigenvector of the
// 2x2 antenna matrix; for a window of a few SFTs of one detector the matrix is
// nearly singular (A B / D up to ~1e7), and any sum rounded to FP32 loses
// ~eps_32 sqrt(AB/D) of relative accuracy in 2F.  The per-cell coefficient
// step marks cells with AB/D > kCondThreshold (Coef.valid = 2); these are
// rare (well below 1% of the cells of the workloads) and always short
// windows in practice.  The fast kernels leave them out, and this file:
//   1. compacts the marked cells into a list in a deterministic order: the
//      coefficient kernels set one bit per marked entry; per-unit counts of
//      the bits, one exclusive scan, ordered writes;
//   2. recomputes each listed cell for every template from the definition
//      over its window (Sec. 2: windowed sums, Eq. F_FaFb) in float-float
//      arithmetic (a value is an unevaluated pair of FP32 numbers, ~2^-47
//      relative per operation; GB300 runs FP64 at 1/64 of the FP32 rate),
//      with D = A B - C^2 and the numerator of 2F formed in float-float too,
//      writes its 2F and adds it to per-block reduction partials kept in
//      their own slots, merged by the final reduction.
#include <math.h>

#include "fmap_batch.cuh"
#include "fmap_device.cuh"

namespace fmap {

constexpr int kFlagBlock = 1024;
constexpr int kFixThreads = 128;
static_assert(kFixPerSlot == kFixThreads, "one entry per thread in a slot of the cell mode");
constexpr int kFixWeights = 256;

// Per unit of kFlagUnit entries: the number of entries marked in the
// bitmask (valid == 2), from the unit's kFlagUnit / 32 words.
constexpr int kFlagWords = kFlagUnit / 32;
static_assert(kFlagWords <= kFlagBlock, "one word per thread");
__device__ __forceinline__ void flag_count_body(const uint32_t* __restrict__ bits, int64_t n_entries, int32_t* __restrict__ blockcnt,
    const uint3 bid, const dim3 gdim) {
  __shared__ int32_t warp_cnt[kFlagBlock / 32];
  const int tid = threadIdx.x;
  const unsigned c = tid < kFlagWords ? (unsigned)__popc(bits[(int64_t)bid.x * kFlagWords + tid]) : 0u;
  const unsigned wsum = __reduce_add_sync(0xffffffffu, c);
  if ((tid & 31) == 0) warp_cnt[tid >> 5] = (int32_t)wsum;
  __syncthreads();
  if (tid < 32) {
    const unsigned t = __reduce_add_sync(0xffffffffu, (unsigned)warp_cnt[tid]);
    if (tid == 0) blockcnt[bid.x] = (int32_t)t;
  }
}

__global__ void __launch_bounds__(kFlagBlock)
k_flag_count(const uint32_t* __restrict__ bits, int64_t n_entries, int32_t* __restrict__ blockcnt) {
  flag_count_body(bits, n_entries, blockcnt, blockIdx, gridDim);
}

// Exclusive scan of the block counts (one block); total into *n_flag.
__device__ __forceinline__ void flag_scan_body(int32_t* __restrict__ blockcnt, int64_t n_blocks, int32_t* __restrict__ n_flag,
    const uint3 bid, const dim3 gdim) {
  __shared__ int32_t warp_sum[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < n_blocks; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const int32_t v = i < n_blocks ? blockcnt[i] : 0;
    int32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int32_t w = warp_sum[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += y;
      }
      warp_sum[lane] = w;  // inclusive
    }
    __syncthreads();
    const int32_t excl = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + x - v;
    if (i < n_blocks) blockcnt[i] = excl;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_flag = carry;
}

__global__ void __launch_bounds__(1024)
k_flag_scan(int32_t* __restrict__ blockcnt, int64_t n_blocks, int32_t* __restrict__ n_flag) {
  flag_scan_body(blockcnt, n_blocks, n_flag, blockIdx, gridDim);
}

// Ordered writes of the marked entries of one unit: each of the unit's words
// (one per thread) places its set bits after the set bits of the words before
// it (an exclusive scan of the words' counts over the block).
__device__ __forceinline__ void flag_write_body(const uint32_t* __restrict__ bits, int64_t n_entries,
             const int32_t* __restrict__ blockoff, int64_t* __restrict__ list,
    const uint3 bid, const dim3 gdim) {
  __shared__ int32_t warp_cnt[kFlagBlock / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t w = (int64_t)bid.x * kFlagWords + tid;
  uint32_t word = tid < kFlagWords ? bits[w] : 0u;
  const int32_t c = __popc(word);
  int32_t x = c;   // inclusive scan within the warp
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_cnt[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int32_t v = warp_cnt[lane];
    int32_t y = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t z = __shfl_up_sync(0xffffffffu, y, d);
      if (lane >= d) y += z;
    }
    warp_cnt[lane] = y - v;   // exclusive over warps
  }
  __syncthreads();
  int64_t off = blockoff[bid.x] + warp_cnt[warp] + (x - c);
  while (word) {
    const int b = __ffs(word) - 1;
    word &= word - 1;
    const int64_t e = w * 32 + b;
    if (e < n_entries && off < n_entries) list[off] = e;   // the list holds at most n_entries
    ++off;
  }
}

__global__ void __launch_bounds__(kFlagBlock)
k_flag_write(const uint32_t* __restrict__ bits, int64_t n_entries,
             const int32_t* __restrict__ blockoff, int64_t* __restrict__ list) {
  flag_write_body(bits, n_entries, blockoff, list, blockIdx, gridDim);
}

// One atom's terms added to the seven float-float sums of a cell: A, B, C
// with weight w^2, Re/Im Fa and Re/Im Fb with weight w (Sec. 2).
__device__ __forceinline__ void fix_add_atom(FF* s, FF w, FF w2, const float* __restrict__ ant,
                                             const float* __restrict__ x, int64_t n, int32_t a) {
  ff_acc(s[0], w2, ant[a]);
  ff_acc(s[1], w2, ant[n + a]);
  ff_acc(s[2], w2, ant[2 * n + a]);
  ff_acc(s[3], w, x[a]);
  ff_acc(s[4], w, x[n + a]);
  ff_acc(s[5], w, x[2 * n + a]);
  ff_acc(s[6], w, x[3 * n + a]);
}

// 2F of a cell from its seven float-float sums (Eq. F_FaFb times two).
// D = A B - C^2 and the numerator B |Fa|^2 + A |Fb|^2 - 2 C Re(Fa Fb*) are
// formed in float-float, so their cancellations cost ~2^-46 A B / D of
// relative accuracy (< 1e-6 at the A B / D ~ 1e7 of the worst cells), then
// divided in FP32.  *ok: at least two atoms and D > 0 (the sign of a
// normalised pair is the sign of its high part).
__device__ __forceinline__ float fix_two_f(const FF* s, int32_t count, bool* ok) {
  const FF D = ff_sub(ff_mul(s[0], s[1]), ff_mul(s[2], s[2]));
  *ok = count >= 2 && D.h > 0.0f;
  if (!*ok) return 0.0f;
  const FF fa2 = ff_add(ff_mul(s[3], s[3]), ff_mul(s[4], s[4]));
  const FF fb2 = ff_add(ff_mul(s[5], s[5]), ff_mul(s[6], s[6]));
  const FF fab = ff_add(ff_mul(s[3], s[5]), ff_mul(s[4], s[6]));
  const FF c2 = {2.0f * s[2].h, 2.0f * s[2].l};
  const FF num = ff_sub(ff_add(ff_mul(s[1], fa2), ff_mul(s[0], fb2)), ff_mul(c2, fab));
  return 2.0f * (num.h / D.h);
}

// Float-float recomputation of listed entries.  Entry = cell (shared antenna:
// every template) or template * cells + cell (per-template antenna: that
// template).  Block (b, y): the entries of slot b (fix_slot_range), templates
// y*128 + tid; the window's weights (w, w^2) are evaluated once per block in
// FP64 and shared as float pairs.
__device__ __forceinline__ void fixup_body(const int64_t* __restrict__ list, const int32_t* __restrict__ n_flag, int32_t G,
        int32_t shared_antenna, const int32_t* __restrict__ rel_t,
        const int64_t* __restrict__ t_base, int32_t n_sft, fmap_grid g, const int64_t* __restrict__ ax, const float2* __restrict__ wtab, int32_t n_tab,
        const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
        const float* __restrict__ antenna, const float* __restrict__ fafb, int32_t n_templates,
        float* __restrict__ map, Partial* __restrict__ parts, int64_t stride, int64_t slot0,
        Coef* __restrict__ coef, const uint3 bid, const dim3 gdim) {
  __shared__ float4 sw[kFixWeights];   // per atom (w, w^2) as float pairs
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const int64_t cap = shared_antenna ? cells : cells * n_templates;   // list capacity
  const int64_t n = min((int64_t)*n_flag, cap);
  int64_t lo, hi;
  fix_slot_range(bid.x, n, G, n_templates, &lo, &hi);
  const int32_t tq = bid.y * kFixThreads + threadIdx.x;
  const bool active_t = tq < n_templates;
  Partial acc = partial_empty();
  for (int64_t k = lo; k < hi; ++k) {
    const int64_t entry = list[k];
    const int64_t cell = shared_antenna ? entry : entry % cells;
    const int32_t only = shared_antenna ? -1 : (int32_t)(entry / cells);
    const int32_t m = (int32_t)(cell / g.n_tau), nn = (int32_t)(cell % g.n_tau);
    const int32_t i0 = i0tab[m], j = jend[cell];
    const int64_t t0rel = grid_t0(g, ax, m) - *t_base;
    const double tau = (double)grid_tau(g, ax, nn);
    const bool mine = active_t && (only < 0 || only == tq);
    const int32_t ta = shared_antenna ? 0 : tq;
    const float* ant = antenna + (int64_t)ta * 3 * n_sft;
    const float* x = fafb + (int64_t)(active_t ? tq : 0) * 4 * n_sft;
    FF sums[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) sums[q] = FF{0.0f, 0.0f};
    for (int32_t a0 = i0; a0 < j; a0 += kFixWeights) {
      __syncthreads();
      for (int32_t u = threadIdx.x; u < kFixWeights; u += kFixThreads) {
        const int32_t a = a0 + u;
        float4 wv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (a < j) {
          const double d = (double)((int64_t)rel_t[a] - t0rel);
          const double w = g.window == FMAP_RECT ? 1.0
              : g.window == FMAP_TABLE ? tab_weight64(d * tab_scale(n_tab, exp_cut8_of(g), grid_tau(g, ax, nn)), wtab, n_tab)
                                       : exp(-d / tau);
          const FF wf = ff_of(w), w2f = ff_of(w * w);
          wv = make_float4(wf.h, wf.l, w2f.h, w2f.l);
        }
        sw[u] = wv;
      }
      __syncthreads();
      if (mine) {
        const int32_t len = min(kFixWeights, j - a0);
        for (int32_t u = 0; u < len; ++u) {
          const float4 wv = sw[u];
          fix_add_atom(sums, FF{wv.x, wv.y}, FF{wv.z, wv.w}, ant, x, n_sft, a0 + u);
        }
      }
    }
    if (mine) {
      bool ok;
      const float v = fix_two_f(sums, j - i0, &ok);
      if (map) map[(int64_t)tq * cells + cell] = v;
      // the validity decision, recorded once per entry
      if (coef && (only >= 0 || tq == 0)) coef[entry].valid = ok ? 3.0f : 0.0f;
      partial_add(acc, v, (int32_t)cell, ok);
    }
  }
  if (active_t) parts[(int64_t)tq * stride + slot0 + bid.x] = acc;
}

// Few templates (T < kFixCellModeT): threads over the listed entries
// instead of templates.  Block (b, tq): the entries of slot b (about
// kFixPerSlot of them, fix_slot_range) for
// template tq, one thread per entry summing its own window in float-float
// (the windows of ill-conditioned cells are a few SFTs long), then a
// fixed-order block reduction of the thread partials.
__device__ __forceinline__ void fixup_cells_body(const int64_t* __restrict__ list,
        const int32_t* __restrict__ n_flag, int32_t G, int32_t shared_antenna,
        const int32_t* __restrict__ rel_t, const int64_t* __restrict__ t_base, int32_t n_sft,
        fmap_grid g, const int64_t* __restrict__ ax, const float2* __restrict__ wtab, int32_t n_tab, const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
        const float* __restrict__ antenna, const float* __restrict__ fafb, int32_t n_templates,
        float* __restrict__ map, Partial* __restrict__ parts, int64_t stride, int64_t slot0,
        Coef* __restrict__ coef, const TauTab* __restrict__ tauc, int32_t b, int32_t tq) {
  __shared__ Partial scratch[kFixThreads / 32];
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const int64_t cap = shared_antenna ? cells : cells * n_templates;
  const int64_t n = min((int64_t)*n_flag, cap);
  int64_t lo, hi;
  fix_slot_range(b, n, G, n_templates, &lo, &hi);
  const int64_t tb = n_sft > 0 ? *t_base : 0;
  const float* ant = antenna + (int64_t)(shared_antenna ? 0 : tq) * 3 * n_sft;
  const float* x = fafb + (int64_t)tq * 4 * n_sft;
  Partial acc = partial_empty();
  for (int64_t k = lo + threadIdx.x; k < hi; k += kFixThreads) {
    const int64_t entry = list[k];
    const int64_t cell = shared_antenna ? entry : entry % cells;
    if (!shared_antenna && entry / cells != tq) continue;
    const int32_t m = (int32_t)(cell / g.n_tau), nn = (int32_t)(cell % g.n_tau);
    const int32_t i0 = i0tab[m], j = jend[cell];
    const int64_t t0rel = grid_t0(g, ax, m) - tb;
    const int64_t tau = grid_tau(g, ax, nn);
    // Exponential weights along the window as products of per-gap decays,
    // the first one being the decay from t0 to the first atom: for gaps of
    // k < kPowTab whole SFTs the tau's float-float powers of the one-SFT
    // decay (~2^-48), an FP64 exp split into a float pair for other gaps;
    // relative error ~(j - i0) 2^-47.
    const bool ex = g.window == FMAP_EXP;
    const bool tb_win = g.window == FMAP_TABLE;
    const double su = tb_win ? tab_scale(n_tab, exp_cut8_of(g), tau) : 0.0;
    const TauTab* tc = ex && tauc ? tauc + nn : nullptr;
    auto decay = [&](int64_t gap) -> FF {
      const int64_t k = gap / g.t_sft;
      if (tc && k < kPowTab && k * g.t_sft == gap) return FF{tc->pw[0][k].x, tc->pw[0][k].y};
      return ff_of(exp(-(double)gap * (tc ? tc->inv_tau : 1.0 / (double)tau)));
    };
    FF sums[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) sums[q] = FF{0.0f, 0.0f};
    FF w{1.0f, 0.0f};
    if (ex && j > i0) w = decay((int64_t)rel_t[i0] - t0rel);
    for (int32_t a = i0; a < j; ++a) {
      if (ex && a > i0) w = ff_mul(w, decay(rel_t[a] - rel_t[a - 1]));
      if (tb_win) w = ff_of(tab_weight64((double)((int64_t)rel_t[a] - t0rel) * su, wtab, n_tab));
      fix_add_atom(sums, w, ff_mul(w, w), ant, x, n_sft, a);
    }
    bool ok;
    const float v = fix_two_f(sums, j - i0, &ok);
    if (map) map[(int64_t)tq * cells + cell] = v;
    if (coef && (!shared_antenna || tq == 0)) coef[entry].valid = ok ? 3.0f : 0.0f;
    partial_add(acc, v, (int32_t)cell, ok);
  }
  acc = partial_block_reduce<kFixThreads / 32>(acc, scratch);
  if (threadIdx.x == 0) parts[(int64_t)tq * stride + slot0 + b] = acc;
}

__global__ void __launch_bounds__(kFixThreads)
k_fixup_cells(const int64_t* __restrict__ list, const int32_t* __restrict__ n_flag, int32_t G,
              int32_t shared_antenna, const int32_t* __restrict__ rel_t,
              const int64_t* __restrict__ t_base, int32_t n_sft, fmap_grid g, const int64_t* __restrict__ ax, const float2* __restrict__ wtab, int32_t n_tab,
              const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
              const float* __restrict__ antenna, const float* __restrict__ fafb,
              int32_t n_templates, float* __restrict__ map, Partial* __restrict__ parts,
              int64_t stride, int64_t slot0, Coef* __restrict__ coef,
              const TauTab* __restrict__ tauc) {
  fixup_cells_body(list, n_flag, G, shared_antenna, rel_t, t_base, n_sft, g, ax, wtab, n_tab, i0tab, jend, antenna,
                   fafb, n_templates, map, parts, stride, slot0, coef, tauc, blockIdx.x, blockIdx.y);
}

// Fix-up blocks of one plan (the y extent: templates, or template blocks).
int64_t fixup_blocks_y(int32_t n_templates) {
  return n_templates < kFixCellModeT ? n_templates
                                     : (n_templates + kFixThreads - 1) / kFixThreads;
}

__global__ void __launch_bounds__(kFixThreads)
k_fixup(const int64_t* __restrict__ list, const int32_t* __restrict__ n_flag, int32_t G,
        int32_t shared_antenna, const int32_t* __restrict__ rel_t,
        const int64_t* __restrict__ t_base, int32_t n_sft, fmap_grid g, const int64_t* __restrict__ ax, const float2* __restrict__ wtab, int32_t n_tab,
        const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
        const float* __restrict__ antenna, const float* __restrict__ fafb, int32_t n_templates,
        float* __restrict__ map, Partial* __restrict__ parts, int64_t stride, int64_t slot0,
        Coef* __restrict__ coef) {
  fixup_body(list, n_flag, G, shared_antenna, rel_t, t_base, n_sft, g, ax, wtab, n_tab, i0tab, jend, antenna, fafb, n_templates, map, parts, stride, slot0, coef, blockIdx, gridDim);
}

cudaError_t launch_flag_and_fixup(fmap_plan_s* p, const fmap_atoms* a, float* d_2F,
                                  cudaStream_t s) {
  const int64_t cells = (int64_t)p->grid.n_t0 * p->grid.n_tau;
  const int64_t n_ant = a->shared_antenna ? 1 : p->n_templates;
  const int64_t n_entries = cells * n_ant;
  if (n_entries == 0 || p->n_templates == 0) return cudaSuccess;
  const int64_t n_blocks = (n_entries + kFlagUnit - 1) / kFlagUnit;
  k_flag_count<<<(unsigned)n_blocks, kFlagBlock, 0, s>>>(p->ws.flag_bits, n_entries, p->ws.flag_blocks);
  k_flag_scan<<<1, 1024, 0, s>>>(p->ws.flag_blocks, n_blocks, p->ws.n_flag);
  k_flag_write<<<(unsigned)n_blocks, kFlagBlock, 0, s>>>(p->ws.flag_bits, n_entries, p->ws.flag_blocks,
                                                         p->ws.flag_list);
  dim3 grid((unsigned)kFixSlots, (unsigned)fixup_blocks_y(p->n_templates));
  if (p->n_templates < kFixCellModeT)
    k_fixup_cells<<<grid, kFixThreads, 0, s>>>(p->ws.flag_list, p->ws.n_flag, kFixSlots,
                                               a->shared_antenna, p->ws.rel_t, p->ws.t_base,
                                               p->n_sft, p->grid, plan_axes(p), p->ws.wtab, p->n_tab,
                                               p->ws.i0, p->ws.jend,
                                               a->antenna, a->fafb, p->n_templates, d_2F,
                                               p->ws.partials, p->part_stride, p->n_tiles,
                                               p->ws.coef,
                                               p->grid.window == FMAP_EXP ? p->ws.tauc : nullptr);
  else
    k_fixup<<<grid, kFixThreads, 0, s>>>(p->ws.flag_list, p->ws.n_flag, kFixSlots,
                                         a->shared_antenna, p->ws.rel_t, p->ws.t_base, p->n_sft,
                                         p->grid, plan_axes(p), p->ws.wtab, p->n_tab, p->ws.i0, p->ws.jend,
                                         a->antenna, a->fafb,
                                         p->n_templates, d_2F, p->ws.partials, p->part_stride,
                                         p->n_tiles, p->ws.coef);
  p->launches += 4;
  return cudaGetLastError();
}


// ---- persistent multi-instance dispatchers (uneven batches) ----
__global__ void __launch_bounds__(kFlagBlock) kb_flag_count(const BItem* __restrict__ items,
                                                            BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    flag_count_body(it.flag_bits, it.flag_entries, it.flag_blocks, make_uint3((unsigned)k, 0, 0),
                    dim3(1));
  });
}
__global__ void __launch_bounds__(1024) kb_flag_scan(const BItem* __restrict__ items, BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t) {
    flag_scan_body(it.flag_blocks, (it.flag_entries + kFlagUnit - 1) / kFlagUnit, it.n_flag,
                   make_uint3(0, 0, 0), dim3(1));
  });
}
__global__ void __launch_bounds__(kFlagBlock) kb_flag_write(const BItem* __restrict__ items,
                                                            BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    flag_write_body(it.flag_bits, it.flag_entries, it.flag_blocks, it.flag_list,
                    make_uint3((unsigned)k, 0, 0), dim3(1));
  });
}
__global__ void __launch_bounds__(kFixThreads) kb_fixup(const BItem* __restrict__ items,
                                                        BUnits u) {
  // unit k: slots [sg * kFixSlotsPerUnit, ...) of template (block) y
  constexpr int kGroups = kFixSlots / kFixSlotsPerUnit;
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    const int32_t sg = (int32_t)(k % kGroups), y = (int32_t)(k / kGroups);
    for (int q = 0; q < kFixSlotsPerUnit; ++q) {
      const int32_t b = sg * kFixSlotsPerUnit + q;
      if (it.T < kFixCellModeT)
        fixup_cells_body(it.flag_list, it.n_flag, kFixSlots, it.shared, it.rel_t, it.t_base,
                         it.n_sft, it.g, it.ax, nullptr, 0, it.i0, it.jend, it.antenna, it.fafb, it.T, it.map,
                         it.partials, it.part_stride, it.n_tiles, it.coef,
                         it.g.window == FMAP_EXP ? it.tauc : nullptr, b, y);
      else
        fixup_body(it.flag_list, it.n_flag, kFixSlots, it.shared, it.rel_t, it.t_base, it.n_sft,
                   it.g, it.ax, nullptr, 0, it.i0, it.jend, it.antenna, it.fafb, it.T, it.map, it.partials,
                   it.part_stride, it.n_tiles, it.coef, make_uint3((unsigned)b, (unsigned)y, 0),
                   dim3((unsigned)kFixSlots, (unsigned)((it.T + kFixThreads - 1) / kFixThreads)));
      __syncthreads();   // the bodies' shared scratch is reused by the next slot
    }
  });
}
const void* batch_kernel_fixup(int phase) {
  switch (phase) {
    case BP_FLAG_COUNT: return (const void*)kb_flag_count;
    case BP_FLAG_SCAN: return (const void*)kb_flag_scan;
    case BP_FLAG_WRITE: return (const void*)kb_flag_write;
    case BP_FIXUP: return (const void*)kb_fixup;
  }
  return nullptr;
}

}  // namespace fmap
