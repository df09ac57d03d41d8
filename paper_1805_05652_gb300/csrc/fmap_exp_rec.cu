// Exponential window by the decayed suffix recurrence (plan flag
// FMAP_PLAN_EXP_RECURRENCE).
//
// The exponential weight factorises in t0: for the atoms [i0, j) of a window,
//   sum_a e^{-(t_a - t0)/tau} x_a = e^{-(t_{i0} - t0)/tau} (E[i0] - e^{-(t_j - t_{i0})/tau} E[j]),
//   E[i] = x_i + e^{-(t_{i+1} - t_i)/tau} E[i+1],  E[N] = 0,
// an exact rearrangement of the window sums of Eq. (winexp).  One recurrence
// per (tau, data column) replaces the per-cell sums: O(N_tau N_SFT) work per
// column instead of O(sum of window lengths).  The recurrence runs as a
// parallel backward scan of the affine maps E -> x + rho E in compensated
// FP32 (float pairs, ~2^-44 relative), and E is rounded to FP32 only for the
// per-cell differences, which then carry the same ~1e-7 relative error as the
// rectangular window's prefix differences.
//
// One block per (tau_n, group of templates): for each template of the group
// the block scans the 4 data columns (read from the chunk-major copy with the
// gaps between atoms; the decays come from the per-tau table of powers of
// the one-SFT decay) into shared memory and evaluates the column of cells
// (t0_m, tau_n) for every m.  Blocks run tau-fastest, so the blocks writing
// neighbouring tau of the same map rows run together and their stores merge
// in L2.
#include <math.h>

#include "fmap_batch.cuh"
#include "fmap_device.cuh"

namespace fmap {

constexpr int kRecThreads = 256;
constexpr int kRecChunk = 8;        // SFTs of data prefetched per serial run of the scan
constexpr int kRecMaxSft = 9000;    // one template's suffix sums in shared memory (144 KB)

struct __align__(16) CellRec {
  int32_t i0, j;
  float pre, tail;
  Coef cf;
};

constexpr size_t kRecSmemCap = 220 * 1024;

// Shared memory of the recurrence: one template's suffix sums, plus the
// staged per-cell records of one tau when they fit.
__host__ __device__ __forceinline__ size_t rec_smem_base(int32_t n_sft) {
  return sizeof(float) * 4 * ((size_t)n_sft + 1) + 16;
}
// Blocks of the recurrence an SM holds with a given dynamic shared memory
// (three at most: the registers of 3 x 256 threads).
__host__ __device__ __forceinline__ int rec_blocks_per_sm(size_t smem) {
  const size_t per_sm = 227 * 1024;
  const size_t k = per_sm / (smem + 1024);
  return (int)(k < 3 ? k : 3);
}
// Staged only for blocks that run two or more templates (a single template
// reads each record once), and only when the staging's shared memory costs
// no resident block (long data sets: the suffix rows alone take 80 KB at
// 5000 SFTs, and with the records an SM would hold one block instead of
// two; recomputing a record per template is cheaper than that).
__host__ __device__ __forceinline__ bool rec_stage_cells(int32_t n_sft, int32_t n_t0, int32_t tpb) {
  const size_t base = rec_smem_base(n_sft), with = base + sizeof(CellRec) * (size_t)n_t0;
  return tpb >= 2 && with <= kRecSmemCap && rec_blocks_per_sm(with) >= rec_blocks_per_sm(base);
}

__device__ __forceinline__ float rec_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// NT = the plan's scan width: threads of the block and width of the
// chunk-major copy.
template <int NT>
__device__ __forceinline__ void exp_rec_body(const int32_t* __restrict__ rel_t, const int64_t* __restrict__ t_base, int32_t n,
          fmap_grid g, const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
          const Coef* __restrict__ coef, int32_t shared_antenna, const float4* __restrict__ perm_x,
          const int32_t* __restrict__ perm_gap, const TauTab* __restrict__ tauc,
          const int64_t* __restrict__ ax, int32_t n_templates, int32_t n_groups,
          float* __restrict__ map, Partial* __restrict__ parts, int64_t stride,
    const uint3 bid, const dim3 gdim) {
  extern __shared__ __align__(16) float s_dyn[];
  float* s_e = s_dyn;                  // [4][n + 1] suffix sums of one template
  // per cell (t0_m, tau_n): the window [i0, j), prefactor, tail factor and the
  // 2F coefficients -- the same for every template, so staged once
  CellRec* s_cell = (CellRec*)(s_e + 4 * ((int64_t)n + 1));
  __shared__ float sR[2][NT / 32];
  __shared__ float sS[4][2][NT / 32];
  __shared__ Partial scratch[NT / 32];
  const int ni = bid.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TauTab* tt = tauc + ni;
  const int64_t np1 = (int64_t)n + 1;
  // Decay after atom i: gaps of k whole SFTs from the tau's table of
  // float-float powers of the one-SFT decay, other gaps by FP64 exp; the gaps
  // come from the chunk-major copy with the data.
  const float inv_tsft = 1.0f / (float)g.t_sft;
  const double inv_tau = tt->inv_tau;
  const int C = (n + NT - 1) / NT;
  const int s0 = min(n, tid * C), e0 = min(n, s0 + C);
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const float c2 = tt->c2[0];
  const bool short_cut = exp_cut8_of(g) < 24;   // window cut before 3 tau
  const int64_t tb = n > 0 ? *t_base : 0;
  // Per cell (t0_m, tau_n): the window, its prefactor and tail factor and the
  // coefficients; staged once per block when they fit, else recomputed per
  // template (large n_sft x n_t0).
  auto cell_rec = [&](int32_t m) {
    const int64_t cell = (int64_t)m * g.n_tau + ni;
    CellRec r;
    r.i0 = i0tab[m];
    r.j = jend[cell];
    r.pre = 0.0f;
    r.tail = 0.0f;
    if (r.j > r.i0) {
      const int64_t t0rel = grid_t0(g, ax, m) - tb;
      const int64_t d0 = (int64_t)rel_t[r.i0] - t0rel;
      r.pre = d0 == 0 ? 1.0f : rec_ex2(c2 * (float)d0);
      if (r.j < n) {
        // Approximate FP32 exp2 for the tail: ~e^{-3} of the window sum for
        // the default 3 tau cut.  Windows cut before 3 tau make it large,
        // where the difference E[i0] - tail E[j] loses 1 / (1 - tail): there a
        // tail above 1/2 comes from the correctly rounded-to-1-ulp exp2f.
        // (An FP64 exp here, even behind a branch never taken, slowed this
        // kernel by 12 %.)
        const int32_t dj = rel_t[r.j] - rel_t[r.i0];
        r.tail = rec_ex2(c2 * (float)dj);
        if (short_cut && r.tail > 0.5f) r.tail = exp2f(c2 * (float)dj);
      }
    }
    r.cf = coef[cell];
    return r;
  };
  const bool stage = rec_stage_cells(n, g.n_t0, (n_templates + n_groups - 1) / n_groups);
  if (stage)
    for (int32_t m = tid; m < g.n_t0; m += NT) s_cell[m] = cell_rec(m);
  const int32_t t_lo = (int32_t)((int64_t)bid.y * n_templates / n_groups);
  const int32_t t_hi = (int32_t)((int64_t)(bid.y + 1) * n_templates / n_groups);
  for (int32_t tq = t_lo; tq < t_hi; ++tq) {
    __syncthreads();   // records staged; previous template's cells done with s_e
    const float4* x = perm_x + (int64_t)tq * perm_entries(n, NT);   // chunk-major data rows
    // phase 1: this thread's chunk as one affine map, E[s0] = S + R E[e0],
    // by the compensated recurrence (folded back every kRecChunk atoms); the
    // data of each run of kRecChunk SFTs is loaded before its serial chain,
    // and positions past the chunk's end are identity steps (x = 0, r = 1)
    float Rh = 1.0f, Rc = 0.0f, Sh[4] = {0.f, 0.f, 0.f, 0.f}, Sc[4] = {0.f, 0.f, 0.f, 0.f};
    float xv[kRecChunk][4];
    int32_t gq[kRecChunk];
    auto load_chunk = [&](int b0) {
#pragma unroll
      for (int q = 0; q < kRecChunk; ++q) {
        const int i = b0 + q;
        const int64_t o = (int64_t)(i - s0) * NT + tid;
        const float4 v = (i < e0) ? __ldg(x + o) : make_float4(0.f, 0.f, 0.f, 0.f);
        gq[q] = (i < e0) ? __ldg(perm_gap + o) : 0;
        xv[q][0] = v.x;
        xv[q][1] = v.y;
        xv[q][2] = v.z;
        xv[q][3] = v.w;
      }
    };
    // identity past the chunk's end (gap 0 there), 0 after the last atom
    auto decay = [&](int q) -> FF {
      if (gq[q] > 0) return gap_decay(gq[q], g.t_sft, inv_tsft, tt->pw[0], inv_tau);
      return gq[q] < 0 ? FF{0.0f, 0.0f} : FF{1.0f, 0.0f};
    };
    for (int b0 = s0 + ((e0 - s0 - 1) / kRecChunk) * kRecChunk; e0 > s0 && b0 >= s0;
         b0 -= kRecChunk) {
      load_chunk(b0);
#pragma unroll
      for (int q = kRecChunk - 1; q >= 0; --q) {
        const FF r = decay(q);
#pragma unroll
        for (int c = 0; c < 4; ++c) ch_step(r, xv[q][c], Sh[c], Sc[c]);
        ch_mul(r, Rh, Rc);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) ch_norm(Sh[c], Sc[c]);
      ch_norm(Rh, Rc);
    }
    FF R = {Rh, Rc}, S[4] = {{Sh[0], Sc[0]}, {Sh[1], Sc[1]}, {Sh[2], Sc[2]}, {Sh[3], Sc[3]}};
    // phase 2: suffix composition within the warp (self o later)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const FF Ro = ff_shfl_down(R, d);
      FF So[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) So[c] = ff_shfl_down(S[c], d);
      if (lane + d < 32) {
#pragma unroll
        for (int c = 0; c < 4; ++c) S[c] = ff_add(S[c], ff_mul(R, So[c]));
        R = ff_mul(R, Ro);
      }
    }
    FF hR = ff_shfl_down(R, 1), hS[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) hS[c] = ff_shfl_down(S[c], 1);
    if (lane == 31) {
      hR = {1.0f, 0.0f};
#pragma unroll
      for (int c = 0; c < 4; ++c) hS[c] = {0.0f, 0.0f};
    }
    if (lane == 0) {
      sR[0][warp] = R.h;
      sR[1][warp] = R.l;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        sS[c][0][warp] = S[c].h;
        sS[c][1][warp] = S[c].l;
      }
    }
    __syncthreads();
    // later warps applied to E[N] = 0
    FF lS[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int v = NT / 32 - 1; v > warp; --v) {
      const FF Rv = {sR[0][v], sR[1][v]};
#pragma unroll
      for (int c = 0; c < 4; ++c) lS[c] = ff_add({sS[c][0][v], sS[c][1][v]}, ff_mul(Rv, lS[c]));
    }
    float eh[4], ec[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const FF e = ff_add(hS[c], ff_mul(hR, lS[c]));
      eh[c] = e.h;
      ec[c] = e.l;
    }
    // phase 3: recompute the chunk from its carry and keep E (rounded) in smem
    for (int b0 = s0 + ((e0 - s0 - 1) / kRecChunk) * kRecChunk; e0 > s0 && b0 >= s0;
         b0 -= kRecChunk) {
      load_chunk(b0);
#pragma unroll
      for (int q = kRecChunk - 1; q >= 0; --q) {
        const int i = b0 + q;
        const FF r = decay(q);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          ch_step(r, xv[q][c], eh[c], ec[c]);
          if (i < e0) s_e[c * np1 + i] = eh[c] + ec[c];
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) ch_norm(eh[c], ec[c]);
    }
    if (tid < 4) s_e[tid * np1 + n] = 0.0f;
    __syncthreads();
    // cells (t0_m, tau_n), all m
    Partial acc = partial_empty();
    for (int32_t m = tid; m < g.n_t0; m += NT) {
      const int64_t cell = (int64_t)m * g.n_tau + ni;
      const CellRec r = stage ? s_cell[m] : cell_rec(m);
      const Coef cf = shared_antenna ? r.cf : coef[(int64_t)tq * cells + cell];
      float f[4] = {0.f, 0.f, 0.f, 0.f};
      if (r.j > r.i0) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          f[c] = r.pre * fmaf(-r.tail, s_e[c * np1 + r.j], s_e[c * np1 + r.i0]);
      }
      const float v = two_f(cf, f[0], f[1], f[2], f[3]);
      const bool ok = cf.valid == 1.0f;
      if (map && cf.valid != 2.0f) map[(int64_t)tq * cells + cell] = ok ? v : 0.0f;
      partial_add(acc, v, (int32_t)cell, ok);
    }
    acc = partial_block_reduce<NT / 32>(acc, scratch);
    if (tid == 0) parts[(int64_t)tq * stride + ni] = acc;
  }
}

template <int NT>
__global__ void __launch_bounds__(NT)
k_exp_rec(const int32_t* __restrict__ rel_t, const int64_t* __restrict__ t_base, int32_t n,
          fmap_grid g, const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
          const Coef* __restrict__ coef, int32_t shared_antenna, const float4* __restrict__ perm_x,
          const int32_t* __restrict__ perm_gap, const TauTab* __restrict__ tauc,
          const int64_t* __restrict__ ax, int32_t n_templates,
          int32_t n_groups, float* __restrict__ map, Partial* __restrict__ parts, int64_t stride) {
  exp_rec_body<NT>(rel_t, t_base, n, g, i0tab, jend, coef, shared_antenna, perm_x, perm_gap, tauc, ax,
               n_templates, n_groups, map, parts, stride, blockIdx, gridDim);
}

bool exp_rec_supported(int32_t n_sft, int32_t) { return n_sft <= kRecMaxSft; }

cudaError_t launch_exp_rec(fmap_plan_s* p, const fmap_atoms* a, float* d_2F, cudaStream_t s,
                           int64_t* tiles_used) {
  const fmap_grid& g = p->grid;
  *tiles_used = 0;
  if ((int64_t)g.n_t0 * g.n_tau == 0 || p->n_templates == 0) return cudaSuccess;
  *tiles_used = g.n_tau;
  p->tiles = TileGeom{0, g.n_t0, 1, 1, g.n_tau};   // one tau column per tile
  // split the templates over enough blocks to fill the GPU a few times
  const int64_t want = (int64_t)p->n_sm * 4;
  const int32_t groups = (int32_t)std::max<int64_t>(
      1, std::min<int64_t>(p->n_templates, (want + g.n_tau - 1) / g.n_tau));
  const size_t smem =
      exp_rec_smem(p->n_sft, g.n_t0, (p->n_templates + groups - 1) / groups);
  dim3 grid((unsigned)g.n_tau, (unsigned)groups);
  auto run = [&](auto kern, int nt) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, nt, smem, s>>>(p->ws.rel_t, p->ws.t_base, p->n_sft, g, p->ws.i0, p->ws.jend,
                                p->ws.coef, a->shared_antenna, p->ws.perm_x, p->ws.perm_gap,
                                p->ws.tauc, plan_axes(p), p->n_templates, groups, d_2F,
                                p->ws.partials, p->part_stride);
  };
  switch (p->lanes) {
    case 64: run(k_exp_rec<64>, 64); break;
    case 128: run(k_exp_rec<128>, 128); break;
    default: run(k_exp_rec<256>, 256); break;
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
    exp_rec_body<NT>(it.rel_t, it.t_base, it.n_sft, it.g, it.i0, it.jend, it.coef, it.shared,
                     it.perm_x, it.perm_gap, it.tauc, it.ax, it.T, it.groups, it.map, it.partials,
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
size_t exp_rec_smem(int32_t n_sft, int32_t n_t0, int32_t tpb) {
  return rec_smem_base(n_sft) +
         (rec_stage_cells(n_sft, n_t0, tpb) ? sizeof(CellRec) * (size_t)n_t0 : 0);
}

}  // namespace fmap
