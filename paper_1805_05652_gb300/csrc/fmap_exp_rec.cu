// Exponential window by the decayed suffix recurrence (plan flag
// FMAP_PLAN_EXP_RECURRENCE).
//
// The exponential weight factorises in t0: for the atoms [i0, j) of a window,
//   sum_a e^{-(t_a - t0)/tau} x_a = e^{-(t_{i0} - t0)/tau} (E[i0] - e^{-(t_j - t_{i0})/tau} E[j]),
//   E[i] = x_i + e^{-(t_{i+1} - t_i)/tau} E[i+1],  E[N] = 0,
// an exact rearrangement of the window sums of Eq. (winexp).  One recurrence
// per (tau, data column) replaces the per-cell sums: O(N_tau N_SFT) work per
// column instead of O(sum of window lengths).  The recurrence runs as a
// parallel backward scan of the affine maps E -> x + rho E.  What spans the
// data set -- the decay products and the composition of the chunks' maps,
// whose errors would otherwise accumulate over up to N_SFT steps -- runs in
// compensated FP32 (float pairs, ~2^-44 relative); the chunk-local sums (at
// most C = 21..35 terms at 5000..9000 SFTs) run in plain FP32, and E is formed
// in FP32 as E = L + Q E[chunk end].  A chunk-local error is at most ~C ulp of
// the chunk's own partial sums, small against E where the window is long
// (slow decay) and limited to the few undecayed terms where it is short:
// emulated on the 5000-SFT workload (every tau class, the cells outside the
// fix-up), the worst relative 2F error is 1.7e-6 against 1.2e-6 for
// compensated chunk sums.
//
// One block per (tau_n, group of templates); each thread owns a chunk of
// atoms (odd length C, read from the chunk-major copy).  Per template of the
// group:
//   1. the chunk-local suffix sums L[i] (E with E[chunk end] = 0) of the 4
//      data columns, one FP32 FMA per atom and column (at most C terms; see
//      below); on the first template also the products Q[i] of the decays
//      from atom i to the chunk's end, in float-float (the same for every
//      template, kept in shared memory) and the chunk's product R;
//   2. the carries E[chunk end] by a suffix composition of the chunks'
//      (L[s0], R) maps, in float-float, within the warp and over the warps;
//   3. E[i] = L[i] + Q[i] E[chunk end] in place (one FMA per column, where
//      recomputing the chunk from its carry would repeat step 1);
//   4. the column of cells (t0_m, tau_n) for every m from E, with the
//      window records (i0, j, prefactor, tail factor; and the coefficients
//      when the antenna is shared) computed on the block's first template and
//      re-read from a tau-major array on the others (the groups of one tau
//      each write the same values there).
// Blocks run tau-fastest, so the blocks writing neighbouring tau of the same
// map rows run together and their stores merge in L2.
#include <math.h>

#include <algorithm>
#include <cmath>

#include "fmap_batch.cuh"
#include "fmap_device.cuh"

namespace fmap {

constexpr int kRecChunk = 8;        // SFTs of data prefetched per serial run of the scan
constexpr int kRecMaxGroups = 32;   // template groups per tau (blocks per tau)
constexpr int kRecMaxSft = 9000;    // one template's suffix sums in shared memory (180 KB)

// Shared memory of the recurrence: E of one template (4 columns) and Q.
__host__ __device__ __forceinline__ size_t rec_smem_base(int32_t n_sft) {
  return sizeof(float) * 5 * ((size_t)n_sft + 1) + 16;
}

__device__ __forceinline__ float rec_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// NT = the plan's scan width: threads of the block and width of the
// chunk-major copy; U = cells a thread loads ahead.
template <int NT, int U>
__device__ __forceinline__ void exp_rec_body(const int32_t* __restrict__ rel_t, const int64_t* __restrict__ t_base, int32_t n,
          fmap_grid g, const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
          const Coef* __restrict__ coef, int32_t shared_antenna, const float4* __restrict__ perm_x,
          const int32_t* __restrict__ perm_gap, float4* __restrict__ recs,
          float* __restrict__ rdec, const TauTab* __restrict__ tauc,
          const int64_t* __restrict__ ax, int32_t n_templates, int32_t n_groups,
          float* __restrict__ map, Partial* __restrict__ parts, int64_t stride,
    const uint3 bid, const dim3 gdim) {
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) float s_dyn[];
  const int64_t np1 = (int64_t)n + 1;
  // [n + 1] L, then E, of one template: the 4 data columns of an atom as one
  // float4 (one 16-byte access where four 4-byte ones would be)
  float4* s_e = reinterpret_cast<float4*>(s_dyn);
  float* s_q = s_dyn + 4 * np1;    // [n] decay product from atom i to its chunk's end
  __shared__ float sR[2][NW];      // each warp's product of its chunks' R
  __shared__ float sS[4][2][NW];   // each warp's composed S (per template)
  __shared__ float sK[4][2][NW];   // E at each warp's end (per template)
  __shared__ Partial scratch[2 * NW];   // the block reductions, alternately
  const int ni = bid.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TauTab* tt = tauc + ni;
  // Decay after atom i: gaps of k whole SFTs from the tau's table of
  // float-float powers of the one-SFT decay, other gaps by FP64 exp; the gaps
  // come from the chunk-major copy with the data.
  const float inv_tsft = 1.0f / (float)g.t_sft;
  const double inv_tau = tt->inv_tau;
  const int C = (int)scan_chunk(n, NT);
  const int s0 = min(n, tid * C), e0 = min(n, s0 + C);
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const float c2 = tt->c2[0];
  const bool short_cut = exp_cut8_of(g) < 24;   // window cut before 3 tau
  const int64_t tb = n > 0 ? *t_base : 0;
  // 0 after the last atom
  int32_t gq[kRecChunk];
  auto decay = [&](int32_t gap) -> FF {
    if (gap > 0) return gap_decay(gap, g.t_sft, inv_tsft, tt->pw[0], inv_tau);
    return gap < 0 ? FF{0.0f, 0.0f} : FF{1.0f, 0.0f};
  };
  const int b_last = s0 + ((e0 - s0 - 1) / kRecChunk) * kRecChunk;   // last run's start
  // window records of tau_n, and coefficients (shared antenna); the array is
  // absent (null) in single-template plans
  float4* rec_a = recs ? recs + (int64_t)ni * g.n_t0 : nullptr;
  float4* rec_c = recs ? recs + cells + (int64_t)ni * g.n_t0 : nullptr;
  // FP32 decays of tau_n in the chunk-major order (absent: computed from the
  // gaps every template)
  float* rd = rdec ? rdec + (int64_t)ni * perm_entries(n, NT) : nullptr;
  const int32_t t_lo = (int32_t)((int64_t)bid.y * n_templates / n_groups);
  const int32_t t_hi = (int32_t)((int64_t)(bid.y + 1) * n_templates / n_groups);
  FF R{1.0f, 0.0f};   // the chunk's product of decays (from the first template on)
  for (int32_t tq = t_lo; tq < t_hi; ++tq) {
    const bool first = tq == t_lo;
    // (the previous template's cells are done with s_e: its block reduction
    // passed a barrier after every warp's cells)
    const float4* x = perm_x + (int64_t)tq * perm_entries(n, NT);   // chunk-major data rows
    // 1. chunk-local suffix sums L[i] in plain FP32 (and on the first
    // template the decay products Q[i] in float-float); the data of each run
    // of kRecChunk SFTs is loaded before its serial chain
    float L[4] = {0.f, 0.f, 0.f, 0.f};
    float Qh = 1.0f, Qc = 0.0f;
    float xv[kRecChunk][4];
    const bool cached = rd && !first;   // decays from the first template's pass
    for (int b0 = b_last; e0 > s0 && b0 >= s0; b0 -= kRecChunk) {
#pragma unroll
      for (int q = 0; q < kRecChunk; ++q) {
        const int i = b0 + q;
        const int64_t o = (int64_t)(i - s0) * NT + tid;
        const float4 v = (i < e0) ? __ldg(x + o) : make_float4(0.f, 0.f, 0.f, 0.f);
        // gq holds the gap, or the cached decay's bits (written by this same
        // thread: a plain load)
        gq[q] = (i < e0) ? (cached ? __float_as_int(rd[o]) : __ldg(perm_gap + o)) : 0;
        xv[q][0] = v.x;
        xv[q][1] = v.y;
        xv[q][2] = v.z;
        xv[q][3] = v.w;
      }
#pragma unroll
      for (int q = kRecChunk - 1; q >= 0; --q) {
        // (only the run at the chunk's end is partial: the same for the
        // warp's lanes but the last thread's)
        if (b0 + q >= e0) continue;
        float rh;
        if (cached) {
          rh = __int_as_float(gq[q]);
        } else {
          const FF r = decay(gq[q]);
          rh = r.h;
          if (first) {
            ch_mul(r, Qh, Qc);
            s_q[b0 + q] = Qh + Qc;
            if (rd) rd[(int64_t)(b0 + q - s0) * NT + tid] = r.h;
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) L[c] = fmaf(rh, L[c], xv[q][c]);
        s_e[b0 + q] = make_float4(L[0], L[1], L[2], L[3]);
      }
      if (first) ch_norm(Qh, Qc);
    }
    if (first) R = {Qh, Qc};
    // 2. carries: suffix composition of the chunks' maps E[s0] = S + R E[e0],
    // within the warp (Rw: the product over lanes lane..31), then over the
    // warps (warp 0, lane v = warp v)
    FF S[4] = {{L[0], 0.f}, {L[1], 0.f}, {L[2], 0.f}, {L[3], 0.f}};
    FF Rw = R;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const FF Ro = ff_shfl_down(Rw, 1 << k);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const FF So = ff_shfl_down(S[c], 1 << k);
        if (lane + (1 << k) < 32) S[c] = ff_fma_sum(S[c], Rw, So);
      }
      if (lane + (1 << k) < 32) Rw = ff_mul(Rw, Ro);
    }
    FF hR = ff_shfl_down(Rw, 1), hS[4];
    if (lane == 31) hR = {1.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      hS[c] = ff_shfl_down(S[c], 1);
      if (lane == 31) hS[c] = {0.0f, 0.0f};
    }
    if (lane == 0) {
      sR[0][warp] = Rw.h;
      sR[1][warp] = Rw.l;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        sS[c][0][warp] = S[c].h;
        sS[c][1][warp] = S[c].l;
      }
    }
    __syncthreads();
    if (warp == 0) {
      FF Rv = lane < NW ? FF{sR[0][lane], sR[1][lane]} : FF{1.0f, 0.0f};
      FF Sv[4];
#pragma unroll
      for (int c = 0; c < 4; ++c)
        Sv[c] = lane < NW ? FF{sS[c][0][lane], sS[c][1][lane]} : FF{0.0f, 0.0f};
#pragma unroll
      for (int k = 0; (1 << k) < NW; ++k) {
        const FF Ro = ff_shfl_down(Rv, 1 << k);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const FF So = ff_shfl_down(Sv[c], 1 << k);
          if (lane + (1 << k) < NW) Sv[c] = ff_fma_sum(Sv[c], Rv, So);
        }
        if (lane + (1 << k) < NW) Rv = ff_mul(Rv, Ro);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        FF K = ff_shfl_down(Sv[c], 1);   // E at the end of warp `lane`
        if (lane >= NW - 1) K = {0.0f, 0.0f};
        if (lane < NW) {
          sK[c][0][lane] = K.h;
          sK[c][1][lane] = K.l;
        }
      }
    }
    __syncthreads();
    // 3. E[i] = L[i] + Q[i] E[e0]
    float Ke[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const FF e = ff_fma_sum(hS[c], hR, FF{sK[c][0][warp], sK[c][1][warp]});
      Ke[c] = e.h + e.l;
    }
    for (int i = s0; i < e0; ++i) {
      const float qi = s_q[i];
      float4 e = s_e[i];
      e.x = fmaf(qi, Ke[0], e.x);
      e.y = fmaf(qi, Ke[1], e.y);
      e.z = fmaf(qi, Ke[2], e.z);
      e.w = fmaf(qi, Ke[3], e.w);
      s_e[i] = e;
    }
    if (tid == 0) s_e[n] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    // 4. cells (t0_m, tau_n), all m
    const bool fresh = first || !recs;   // records computed here (no array: one template)
    // U cells per thread at a time: their records (or, when computed here,
    // their window indices and then the atom times those select) are all
    // loaded before any is used, so the loads' latencies overlap
    Partial acc = partial_empty();
    for (int32_t mb = tid; mb < g.n_t0; mb += NT * U) {
      float4 ra[U], rc[U];
      if (fresh) {
        int32_t i0v[U], jv[U], ti[U], tj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int32_t m = mb + u * NT;
          const bool in = m < g.n_t0;
          i0v[u] = in ? i0tab[m] : 0;
          jv[u] = in ? jend[(int64_t)m * g.n_tau + ni] : 0;
          if (shared_antenna) {
            const Coef cf = in ? coef[(int64_t)m * g.n_tau + ni] : Coef{0.f, 0.f, 0.f, 0.f};
            rc[u] = make_float4(cf.k1, cf.beta, cf.k2, cf.valid);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool any = jv[u] > i0v[u];
          ti[u] = any ? rel_t[i0v[u]] : 0;
          tj[u] = any && jv[u] < n ? rel_t[jv[u]] : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          // the window [i0, j), its prefactor and its tail factor
          const int32_t m = mb + u * NT;
          float pre = 0.0f, tail = 0.0f;
          if (jv[u] > i0v[u]) {
            const int64_t d0 = (int64_t)ti[u] - (grid_t0(g, ax, m) - tb);
            pre = d0 == 0 ? 1.0f : rec_ex2(c2 * (float)d0);
            if (jv[u] < n) {
              // Approximate FP32 exp2 for the tail: ~e^{-3} of the window
              // sum for the default 3 tau cut.  Windows cut before 3 tau make
              // it large, where the difference E[i0] - tail E[j] loses 1 / (1
              // - tail): there a tail above 1/2 comes from the correctly
              // rounded-to-1-ulp exp2f.  (An FP64 exp here, even behind a
              // branch never taken, slowed this kernel by 12 %.)
              const float dj = (float)(tj[u] - ti[u]);
              tail = rec_ex2(c2 * dj);
              if (short_cut && tail > 0.5f) tail = exp2f(c2 * dj);
            }
          }
          ra[u] = make_float4(__int_as_float(i0v[u]), __int_as_float(jv[u]), pre, tail);
          if (recs && m < g.n_t0) {   // (read back by this same thread on later templates)
            rec_a[m] = ra[u];
            if (shared_antenna) rec_c[m] = rc[u];
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int32_t m = mb + u * NT;
          const bool in = m < g.n_t0;
          ra[u] = in ? rec_a[m] : make_float4(0.f, 0.f, 0.f, 0.f);
          if (shared_antenna) rc[u] = in ? rec_c[m] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      if (!shared_antenna) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int32_t m = mb + u * NT;
          const Coef cf = m < g.n_t0 ? coef[(int64_t)tq * cells + (int64_t)m * g.n_tau + ni]
                                     : Coef{0.f, 0.f, 0.f, 0.f};
          rc[u] = make_float4(cf.k1, cf.beta, cf.k2, cf.valid);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t m = mb + u * NT;
        if (m >= g.n_t0) break;
        const int64_t cell = (int64_t)m * g.n_tau + ni;
        const int32_t i0 = __float_as_int(ra[u].x), j = __float_as_int(ra[u].y);
        float f[4] = {0.f, 0.f, 0.f, 0.f};
        if (j > i0) {
          const float4 ej = s_e[j], ei = s_e[i0];
          f[0] = ra[u].z * fmaf(-ra[u].w, ej.x, ei.x);
          f[1] = ra[u].z * fmaf(-ra[u].w, ej.y, ei.y);
          f[2] = ra[u].z * fmaf(-ra[u].w, ej.z, ei.z);
          f[3] = ra[u].z * fmaf(-ra[u].w, ej.w, ei.w);
        }
        const Coef cf{rc[u].x, rc[u].y, rc[u].z, rc[u].w};
        const float v = two_f(cf, f[0], f[1], f[2], f[3]);
        const bool ok = cf.valid == 1.0f;
        if (map && cf.valid != 2.0f) map[(int64_t)tq * cells + cell] = ok ? v : 0.0f;
        partial_add(acc, v, (int32_t)cell, ok);
      }
    }
    acc = partial_block_reduce_alt<NW>(acc, scratch, tq - t_lo);
    if (tid == 0) parts[(int64_t)tq * stride + ni] = acc;
  }
}

// MB blocks of 256 threads' register budget per SM, for any width: MB = 3
// where shared memory lets three blocks reside, else 2 (more registers, no
// occupancy lost).
template <int NT, int MB>
__global__ void __launch_bounds__(NT, MB * 256 / NT)
k_exp_rec(const int32_t* __restrict__ rel_t, const int64_t* __restrict__ t_base, int32_t n,
          fmap_grid g, const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
          const Coef* __restrict__ coef, int32_t shared_antenna, const float4* __restrict__ perm_x,
          const int32_t* __restrict__ perm_gap, float4* __restrict__ recs, float* __restrict__ rdec,
          const TauTab* __restrict__ tauc, const int64_t* __restrict__ ax, int32_t n_templates,
          int32_t n_groups, float* __restrict__ map, Partial* __restrict__ parts, int64_t stride) {
  exp_rec_body<NT, MB == 2 ? 4 : 2>(rel_t, t_base, n, g, i0tab, jend, coef, shared_antenna, perm_x, perm_gap, recs,
                   rdec, tauc, ax, n_templates, n_groups, map, parts, stride, blockIdx, gridDim);
}

bool exp_rec_supported(int32_t n_sft, int32_t) { return n_sft <= kRecMaxSft; }

cudaError_t launch_exp_rec(fmap_plan_s* p, const fmap_atoms* a, float* d_2F, cudaStream_t s,
                           int64_t* tiles_used) {
  const fmap_grid& g = p->grid;
  *tiles_used = 0;
  if ((int64_t)g.n_t0 * g.n_tau == 0 || p->n_templates == 0) return cudaSuccess;
  *tiles_used = g.n_tau;
  p->tiles = TileGeom{0, g.n_t0, 1, 1, g.n_tau};   // one tau column per tile
  const size_t smem = exp_rec_smem(p->n_sft, g.n_t0, p->n_templates);
  const bool three = smem + 1024 <= 227 * 1024 / 3;
  // The templates are split into G groups, one block per (tau, group), with
  // G chosen so that the blocks fill whole waves of the resident slots: the
  // step takes about ceil(blocks / slots) block times, and a block's time is
  // its templates plus about 1.5 templates' worth of first-template work
  // (decay products, window records).  Measured on GB300: 1024 templates x
  // 2000 tau, G = 5 is 7 % faster than one block per tau; 16 x 1000, G = 2
  // is 8 % faster.
  const int nt = p->lanes == 64 || p->lanes == 128 ? p->lanes : 256;
  const int64_t per_sm = std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)(three ? 3 : 2) * 256 / nt, (int64_t)2048 / nt,
                            (int64_t)(227 * 1024) / (int64_t)(smem + 1024)}));
  const int64_t slots = (int64_t)p->n_sm * per_sm;
  int32_t groups = 1;
  double best = 0.0;
  for (int32_t G = 1; G <= std::min<int32_t>(p->n_templates, kRecMaxGroups); ++G) {
    const double waves = std::ceil((double)g.n_tau * G / (double)slots);
    const double cost = waves * ((double)((p->n_templates + G - 1) / G) + 1.5);
    if (G == 1 || cost < best) {
      best = cost;
      groups = G;
    }
  }
  dim3 grid((unsigned)g.n_tau, (unsigned)groups);
  auto run = [&](auto kern, int nt) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, nt, smem, s>>>(p->ws.rel_t, p->ws.t_base, p->n_sft, g, p->ws.i0, p->ws.jend,
                                p->ws.coef, a->shared_antenna, p->ws.perm_x, p->ws.perm_gap,
                                p->ws.rec_cells, p->ws.rec_decay, p->ws.tauc, plan_axes(p), p->n_templates, groups, d_2F,
                                p->ws.partials, p->part_stride);
  };
  switch (p->lanes) {
    case 64: three ? run(k_exp_rec<64, 3>, 64) : run(k_exp_rec<64, 2>, 64); break;
    case 128: three ? run(k_exp_rec<128, 3>, 128) : run(k_exp_rec<128, 2>, 128); break;
    default: three ? run(k_exp_rec<256, 3>, 256) : run(k_exp_rec<256, 2>, 256); break;
  }
  p->launches += 1;
  return cudaGetLastError();
}


// ---- persistent multi-instance dispatcher (uneven batches) ----
// (the register budget of 3 blocks of 256 threads per SM, for any width)
template <int NT>
__global__ void __launch_bounds__(NT, 768 / NT) kb_exp_rec(const BItem* __restrict__ items,
                                                        BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    exp_rec_body<NT, 2>(it.rel_t, it.t_base, it.n_sft, it.g, it.i0, it.jend, it.coef, it.shared,
                     it.perm_x, it.perm_gap, it.rec_cells, nullptr, it.tauc, it.ax, it.T, it.groups, it.map, it.partials,
                     it.part_stride,
                     make_uint3((unsigned)(k % it.g.n_tau), (unsigned)(k / it.g.n_tau), 0),
                     dim3((unsigned)it.g.n_tau, (unsigned)it.groups));
  });
}
const void* batch_kernel_exp_rec(int phase, int lanes) {
  if (phase != BP_EXP_REC) return nullptr;
  return lanes == 64 ? (const void*)kb_exp_rec<64>
                     : lanes == 128 ? (const void*)kb_exp_rec<128> : (const void*)kb_exp_rec<256>;
}
size_t exp_rec_smem(int32_t n_sft, int32_t, int32_t) { return rec_smem_base(n_sft); }

}  // namespace fmap
