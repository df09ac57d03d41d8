// Exponential-window F-map (Eq. winexp, cut after 3 tau).
//
// Antenna part (shared by every template of a sky position): A, B, C with the
// squared weight w^2 = e^{-2(t - t0)/tau}, in FP64, from a decayed suffix
// sum per tau:
//     E[i] = x_i + e^{-2(t_{i+1} - t_i)/tau} E[i+1],   E[N] = 0,
//     A(t0, tau) = e^{-2(t_{i0} - t0)/tau} (E[i0] - e^{-2(t_j - t_{i0})/tau} E[j])
// for the window's atoms [i0, j).  The recurrence is contractive, so the
// subtraction loses at most a factor 1/(1 - e^{-6}) of relative accuracy.
// Then D = AB - C^2 in FP64 and the per-cell 2F coefficients.
//
// Data part: Fa, Fb = sum_a w(t_a) X[a, col] over the window, a contraction
// of the weight matrix W[(t0, tau), a] with the 4T data columns.  Here the
// plain CUDA-core form (the paper's brute-force exp kernel, Sec. 3, restated
// with shared-memory staging and one thread per cell): FP32 or FP64
// accumulation.  The tensor-core form lives in fmap_exp_tc.cu.
#include <math.h>

#include <type_traits>

#include "fmap_batch.cuh"
#include "fmap_device.cuh"

namespace fmap {

constexpr int kSufThreads = 256;

// r^k for small k >= 1 by binary powering (relative error ~k ulp).
__device__ __forceinline__ double ipow(double r, int k) {
  double acc = 1.0;
  while (k) {
    if (k & 1) acc *= r;
    r *= r;
    k >>= 1;
  }
  return acc;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Decayed suffix sums of the three antenna rows for one tau, by a parallel
// backward scan of the affine maps E -> x + rho E over the block's threads,
// in float-float arithmetic (the FP32 pipe; GB300's FP64 rate is 1/64 of
// it): E[c * (n + 1) + i] for c = a2, b2, ab and i = 0..n (E[n] = 0), each as
// an (h, l) pair.  E may be in global or shared memory; the block must call
// it together.
// NT = the plan's scan width: the threads of the block and the width of the
// chunk-major copy.
template <int NT>
__device__ __forceinline__ void antenna_suffix(const float4* __restrict__ perm, int32_t n,
                                               const fmap_grid& g,
                                               const TauTab* __restrict__ tt, float2* E,
                                               float (*sR)[NT / 32],
                                               float (*sS)[2][NT / 32]) {
  const double inv_s = 2.0 * tt->inv_tau;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int C = (int)scan_chunk(n, NT);
  const int s0 = min(n, tid * C), e0 = min(n, s0 + C);
  // Decay over one gap: e^{-2 gap / tau}, from the tau's table of powers of
  // the one-SFT decay (FP64 exp off the T_sft lattice).
  const float inv_tsft = 1.0f / (float)g.t_sft;
  auto rho_of_gap = [&](int32_t gap) -> FF {
    return gap_decay(gap, g.t_sft, inv_tsft, tt->pw[1], inv_s);
  };
  // The chunk's atoms (three antenna rows and the gap to the next atom) are
  // read kSufChunk at a time ahead of each serial run, so the chain does not
  // wait on memory per atom; the chunk-major copy makes each of these loads
  // one contiguous 512-byte row per warp.
  constexpr int kSufChunk = 8;
  float xa[kSufChunk][3];
  int32_t gap[kSufChunk];
  auto load_chunk = [&](int b0) {
#pragma unroll
    for (int q = 0; q < kSufChunk; ++q) {
      const int i = b0 + q;
      const bool in = i < e0;
      const float4 v = in ? __ldg(perm + (int64_t)(i - s0) * NT + tid)
                          : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
      xa[q][0] = v.x;
      xa[q][1] = v.y;
      xa[q][2] = v.z;
      gap[q] = __float_as_int(v.w);
    }
  };
  auto rho_q = [&](int q) -> FF { return gap[q] < 0 ? FF{0.0f, 0.0f} : rho_of_gap(gap[q]); };
  // phase 1: compose this thread's chunk: E[s0] = S + R E[e0]
  FF R{1.0f, 0.0f}, S[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int b0 = s0 + ((e0 - s0 - 1) / kSufChunk) * kSufChunk; e0 > s0 && b0 >= s0;
       b0 -= kSufChunk) {
    load_chunk(b0);
#pragma unroll
    for (int q = kSufChunk - 1; q >= 0; --q) {
      if (b0 + q >= e0) continue;
      const FF r = rho_q(q);
#pragma unroll
      for (int c = 0; c < 3; ++c) S[c] = ff_axpy(r, S[c], xa[q][c]);
      R = ff_mul(r, R);
    }
  }
  // phase 2: inclusive suffix composition within the warp (self o later)
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const FF Ro = ff_shfl_down(R, d);
    FF So[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) So[c] = ff_shfl_down(S[c], d);
    if (lane + d < 32) {
#pragma unroll
      for (int c = 0; c < 3; ++c) S[c] = ff_add(S[c], ff_mul(R, So[c]));
      R = ff_mul(R, Ro);
    }
  }
  // exclusive within the warp: composition of lanes lane+1 .. 31
  FF hR = ff_shfl_down(R, 1), hS[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) hS[c] = ff_shfl_down(S[c], 1);
  if (lane == 31) {
    hR = {1.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < 3; ++c) hS[c] = {0.0f, 0.0f};
  }
  if (lane == 0) {
    sR[0][warp] = R.h;
    sR[1][warp] = R.l;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sS[c][0][warp] = S[c].h;
      sS[c][1][warp] = S[c].l;
    }
  }
  __syncthreads();
  // composition of the later warps, applied to E[N] = 0: only its S matters
  FF lS[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int v = NT / 32 - 1; v > warp; --v) {
    const FF Rv{sR[0][v], sR[1][v]};
#pragma unroll
    for (int c = 0; c < 3; ++c) lS[c] = ff_add(FF{sS[c][0][v], sS[c][1][v]}, ff_mul(Rv, lS[c]));
  }
  FF e[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) e[c] = ff_add(hS[c], ff_mul(hR, lS[c]));
  // phase 3: recompute the chunk from its carry E[e0] and store
  const int64_t np1 = (int64_t)n + 1;
  for (int b0 = s0 + ((e0 - s0 - 1) / kSufChunk) * kSufChunk; e0 > s0 && b0 >= s0;
       b0 -= kSufChunk) {
    load_chunk(b0);
#pragma unroll
    for (int q = kSufChunk - 1; q >= 0; --q) {
      const int i = b0 + q;
      if (i >= e0) continue;
      const FF r = rho_q(q);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        e[c] = ff_axpy(r, e[c], xa[q][c]);
        E[c * np1 + i] = make_float2(e[c].h, e[c].l);
      }
    }
  }
  if (tid == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) E[c * np1 + n] = make_float2(0.0f, 0.0f);
  }
}

// Global-memory suffix sums for one tau of a tau chunk (long data sets).
__global__ void __launch_bounds__(kSufThreads)
k_exp_suffix(const float4* __restrict__ perm, const TauTab* __restrict__ tauc, int32_t n,
             fmap_grid g, int32_t n_lo, float2* __restrict__ esuf) {
  static_assert(kSufThreads == kScanLanes, "data sets past shared memory take the widest scan");
  __shared__ float sR[2][kSufThreads / 32];
  __shared__ float sS[3][2][kSufThreads / 32];
  const int ni = blockIdx.x;
  antenna_suffix<kSufThreads>(perm, n, g, tauc + n_lo + ni,
                              esuf + (int64_t)ni * 3 * ((int64_t)n + 1), sR, sS);
}

// Tail factors above this size are taken from FP64 exp as float pairs: the
// window sum E[i0] - tail E[j] then loses 1 / (1 - tail) of relative accuracy
// to the tail's own error, which the ill-conditioned D = AB - C^2 amplifies
// further (windows cut well before 3 tau, or starting in a long gap).
constexpr float kTailExact = 1.0f / 32.0f;

// A, B, C of the cell (t0, tau) from the suffix sums E of its tau, then its
// coefficients; c2 = -2 log2(e) / tau, inv_tau = 1 / tau.  t_i0 and t_j are
// the relative times of atoms i0 and j (read only when the window holds
// atoms, and t_j only when j < n).
__device__ __forceinline__ Coef exp_cell_coef_t(int32_t t_i0, int32_t t_j, int32_t n,
                                                int64_t t0, float c2,
                                                double inv_tau, int32_t i0, int32_t j,
                                                int64_t t_base, const float2* E) {
  const int32_t count = j - i0;
  FF S[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  if (count > 0) {
    const int64_t t0rel = t0 - t_base;
    const int64_t np1 = (int64_t)n + 1;
    // The prefactor scales A, B, C alike (F changes by its relative error
    // only): FP32 exp2 is accurate enough.  The tail is FP32 exp2 while it is
    // small (~e^{-6} of the window sum for the default 3 tau cut), FP64 exp
    // otherwise.
    const int64_t d0 = (int64_t)t_i0 - t0rel;
    const float pre = d0 == 0 ? 1.0f : ex2_approx(c2 * (float)d0);
    FF tail{0.0f, 0.0f};
    if (j < n) {
      const int32_t dj = t_j - t_i0;
      tail.h = ex2_approx(c2 * (float)dj);
      if (tail.h > kTailExact) tail = ff_of(exp(-2.0 * (double)dj * inv_tau));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 a = E[c * np1 + i0], b = E[c * np1 + j];
      S[c] = ff_mul_f(ff_sub(FF{a.x, a.y}, ff_mul(FF{b.x, b.y}, tail)), pre);
    }
  }
  return make_coef_ff(S[0], S[1], S[2], count);
}
__device__ __forceinline__ Coef exp_cell_coef(const int32_t* __restrict__ rel_t, int32_t n,
                                              int64_t t0, float c2,
                                              double inv_tau, int32_t i0, int32_t j,
                                              int64_t t_base, const float2* E) {
  const bool any = j > i0;
  return exp_cell_coef_t(any ? rel_t[i0] : 0, any && j < n ? rel_t[j] : 0, n, t0, c2, inv_tau,
                         i0, j, t_base, E);
}

// cells a thread loads ahead in the antenna kernels (fewer for the narrowest
// scan, whose batch variant runs at the highest occupancy)
template <int NT>
constexpr int cells_in_flight() { return NT >= 128 ? 4 : 2; }

// Fused antenna step for data sets that fit shared memory: one block per
// (tau_n, antenna set) keeps the suffix sums in shared memory and writes the
// coefficients of every cell (t0_m, tau_n).  Blocks run tau-fastest, so their
// strided coefficient stores merge in L2.
template <int NT>
__device__ __forceinline__ void exp_antenna_body(const int32_t* __restrict__ rel_t, const int64_t* __restrict__ t_base, int32_t n,
              fmap_grid g, const float4* __restrict__ perm_ant, const TauTab* __restrict__ tauc,
              const int64_t* __restrict__ ax, const int32_t* __restrict__ i0tab,
              const int32_t* __restrict__ jend, Coef* __restrict__ coef,
              uint32_t* __restrict__ bits, const uint3 bid, const dim3 gdim) {
  extern __shared__ float2 s_E[];
  __shared__ float sR[2][NT / 32];
  __shared__ float sS[3][2][NT / 32];
  const int ni = bid.x, ta = bid.y;
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const TauTab* tt = tauc + ni;
  antenna_suffix<NT>(perm_ant + (int64_t)ta * perm_entries(n, NT), n, g, tt, s_E, sR, sS);
  __syncthreads();
  const int64_t tb = n > 0 ? *t_base : 0;
  // U cells per thread at a time: their window indices, then the atom times
  // those select, are all loaded before any is used, so the loads' latencies
  // overlap.
  constexpr int U = cells_in_flight<NT>();
  for (int32_t m0 = threadIdx.x; m0 < g.n_t0; m0 += NT * U) {
    int32_t i0v[U], jv[U], ti[U], tj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t m = m0 + u * NT;
      const bool in = m < g.n_t0;
      i0v[u] = in ? i0tab[m] : 0;
      jv[u] = in ? jend[(int64_t)m * g.n_tau + ni] : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool any = jv[u] > i0v[u];
      ti[u] = any ? rel_t[i0v[u]] : 0;
      tj[u] = any && jv[u] < n ? rel_t[jv[u]] : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t m = m0 + u * NT;
      if (m < g.n_t0)
        store_coef(coef, bits, (int64_t)ta * cells + (int64_t)m * g.n_tau + ni,
                   exp_cell_coef_t(ti[u], tj[u], n, grid_t0(g, ax, m), tt->c2[1], tt->inv_tau,
                                   i0v[u], jv[u], tb, s_E));
    }
  }
}

template <int NT>
__global__ void __launch_bounds__(NT)
k_exp_antenna(const int32_t* __restrict__ rel_t, const int64_t* __restrict__ t_base, int32_t n,
              fmap_grid g, const float4* __restrict__ perm_ant, const TauTab* __restrict__ tauc,
              const int64_t* __restrict__ ax, const int32_t* __restrict__ i0tab,
              const int32_t* __restrict__ jend, Coef* __restrict__ coef,
              uint32_t* __restrict__ bits) {
  exp_antenna_body<NT>(rel_t, t_base, n, g, perm_ant, tauc, ax, i0tab, jend, coef, bits, blockIdx,
                       gridDim);
}

// Chunk-major copies of one instance's atoms for the scans: entry
// q lanes + t of a set holds atom i = t C + q (zeros past the last atom; lanes
// = the plan's scan width, C = scan_chunk(n, lanes)):
// sets 0..n_ant-1 the antenna rows with the gap to the next atom, sets
// n_ant.. the data rows of each template (when perm_x is given); then the
// per-tau constants (n_tau more entries).
__device__ __forceinline__ void exp_perm_body(const int32_t* __restrict__ rel_t, int32_t n,
                                              int32_t lanes,
                                              const float* __restrict__ antenna, int32_t n_ant,
                                              const float* __restrict__ fafb, int32_t n_x,
                                              float4* __restrict__ perm_ant,
                                              float4* __restrict__ perm_x,
                                              int32_t* __restrict__ perm_gap, const fmap_grid& g,
                                              const int64_t* __restrict__ ax,
                                              TauTab* __restrict__ tauc, int64_t e_begin,
                                              int64_t e_end, int64_t e_step) {
  const int64_t P = perm_entries(n, lanes), C = scan_chunk(n, lanes);
  const int64_t n_copy = P * (int64_t)(n_ant + n_x);
  for (int64_t e = e_begin; e < e_end; e += e_step) {
    if (e >= n_copy) {   // entries past the copies: the per-tau constants
      tau_tab_fill(g, grid_tau(g, ax, e - n_copy), tauc + (e - n_copy));
      continue;
    }
    const int64_t set = e / P, r = e - set * P;
    const int64_t q = r / lanes, t = r - q * lanes;
    const int64_t i = t * C + q;
    const bool in = i < n;
    if (set < n_ant) {
      const float* a = antenna + set * 3 * (int64_t)n;
      float4 v = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
      if (in) {
        const int32_t gap = i + 1 < n ? rel_t[i + 1] - rel_t[i] : -1;
        v = make_float4(a[i], a[n + i], a[2 * (int64_t)n + i], __int_as_float(gap));
      }
      perm_ant[e] = v;
      if (set == 0 && perm_gap) perm_gap[r] = __float_as_int(v.w);
    } else {
      const int64_t tq = set - n_ant;
      const float* x = fafb + tq * 4 * (int64_t)n;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (in) v = make_float4(x[i], x[n + i], x[2 * (int64_t)n + i], x[3 * (int64_t)n + i]);
      perm_x[tq * P + r] = v;
    }
  }
}

__global__ void k_exp_perm(const int32_t* __restrict__ rel_t, int32_t n, int32_t lanes,
                           const float* __restrict__ antenna, int32_t n_ant,
                           const float* __restrict__ fafb, int32_t n_x,
                           float4* __restrict__ perm_ant, float4* __restrict__ perm_x,
                           int32_t* __restrict__ perm_gap, fmap_grid g,
                           const int64_t* __restrict__ ax, TauTab* __restrict__ tauc) {
  const int64_t total = exp_copy_entries(n, lanes, n_ant, n_x, g.n_tau);
  exp_perm_body(rel_t, n, lanes, antenna, n_ant, fafb, n_x, perm_ant, perm_x, perm_gap, g, ax, tauc,
                (int64_t)blockIdx.x * blockDim.x + threadIdx.x, total,
                (int64_t)gridDim.x * blockDim.x);
}

cudaError_t launch_exp_perm(fmap_plan_s* p, const fmap_atoms* a, cudaStream_t s) {
  if ((int64_t)p->grid.n_t0 * p->grid.n_tau == 0) return cudaSuccess;
  const int32_t n_ant = a->shared_antenna ? 1 : p->n_templates;
  const int32_t n_x = p->ws.perm_x ? p->n_templates : 0;
  const int64_t total = exp_copy_entries(p->n_sft, p->lanes, n_ant, n_x, p->grid.n_tau);
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)p->n_sm * 16);
  k_exp_perm<<<blocks, 256, 0, s>>>(p->ws.rel_t, p->n_sft, p->lanes, a->antenna, n_ant, a->fafb, n_x,
                                    p->ws.perm_ant, p->ws.perm_x, p->ws.perm_gap, p->grid,
                                    plan_axes(p), p->ws.tauc);
  p->launches += 1;
  return cudaGetLastError();
}

constexpr int kAntennaSmemMaxSft = 9000;   // 3 x (n + 1) float pairs <= 216 KB

// Per-cell coefficients of the cells of one tau chunk (global suffix sums).
__global__ void k_exp_coef(const int32_t* __restrict__ rel_t, const int64_t* __restrict__ t_base,
                           int32_t n, fmap_grid g, int32_t n_lo, int32_t n_chunk,
                           const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
                           const float2* __restrict__ esuf, const TauTab* __restrict__ tauc,
                           const int64_t* __restrict__ ax, Coef* __restrict__ coef,
                           uint32_t* __restrict__ bits, int64_t e_base) {
  const int64_t total = (int64_t)g.n_t0 * n_chunk;
  const int64_t np1 = (int64_t)n + 1;
  const int64_t tb = n > 0 ? *t_base : 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = c / n_chunk;
    const int32_t nl = (int32_t)(c - m * n_chunk);
    const int64_t nn = n_lo + nl;
    const int64_t cell = m * g.n_tau + nn;
    store_coef(coef, bits, e_base + cell,
               exp_cell_coef(rel_t, n, grid_t0(g, ax, m), tauc[nn].c2[1], tauc[nn].inv_tau,
                             i0tab[m], jend[cell], tb, esuf + (int64_t)nl * 3 * np1));
  }
}

cudaError_t launch_exp_coef(fmap_plan_s* p, const fmap_atoms* a, cudaStream_t s) {
  const fmap_grid& g = p->grid;
  if ((int64_t)g.n_t0 * g.n_tau == 0) return cudaSuccess;
  const int n_ant = a->shared_antenna ? 1 : p->n_templates;
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  if (p->n_sft <= kAntennaSmemMaxSft) {
    const size_t smem = exp_antenna_smem(p->n_sft);
    auto run = [&](auto kern, int nt) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kern<<<dim3((unsigned)g.n_tau, (unsigned)n_ant), nt, smem, s>>>(
          p->ws.rel_t, p->ws.t_base, p->n_sft, g, p->ws.perm_ant, p->ws.tauc, plan_axes(p),
          p->ws.i0, p->ws.jend, p->ws.coef, p->ws.flag_bits);
    };
    switch (p->lanes) {
      case 64: run(k_exp_antenna<64>, 64); break;
      case 128: run(k_exp_antenna<128>, 128); break;
      default: run(k_exp_antenna<256>, 256); break;
    }
    p->launches += 1;
    return cudaGetLastError();
  }
  for (int ta = 0; ta < n_ant; ++ta) {
    const float4* perm = p->ws.perm_ant + (int64_t)ta * perm_entries(p->n_sft, p->lanes);
    for (int32_t lo = 0; lo < g.n_tau; lo += p->tau_chunk) {
      const int32_t len = std::min<int32_t>(p->tau_chunk, g.n_tau - lo);
      if (p->n_sft > 0) {
        k_exp_suffix<<<len, kSufThreads, 0, s>>>(perm, p->ws.tauc, p->n_sft, g, lo, p->ws.esuf);
        p->launches += 1;
      }
      const int64_t total = (int64_t)g.n_t0 * len;
      const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)p->n_sm * 16);
      k_exp_coef<<<blocks, 256, 0, s>>>(p->ws.rel_t, p->ws.t_base, p->n_sft, g, lo, len, p->ws.i0,
                                        p->ws.jend, p->ws.esuf, p->ws.tauc, plan_axes(p),
                                        p->ws.coef, p->ws.flag_bits, ta * cells);
      p->launches += 1;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Plain contraction on the CUDA cores.  Tile = 128 cells: one t0 row m and
// 128 consecutive tau; they share i0, so the tile's atoms are [i0, max j).
// The weights are computed once per (cell, atom) and reused for the TC
// templates of the block; atoms are staged KC at a time in shared memory.
// ---------------------------------------------------------------------------
constexpr int kExpCells = 128;
constexpr int kKC = 32;

int64_t exp_tiles(const fmap_grid& g) {
  return (int64_t)g.n_t0 * ((g.n_tau + kExpCells - 1) / kExpCells);
}

// TAB: the weights come from the window table wtab (n_tab samples; FMAP_TABLE
// grids) instead of the exponential.
template <typename Acc, int TC, bool TAB>
__global__ void __launch_bounds__(kExpCells)
k_exp_plain(const int32_t* __restrict__ rel_t, const int64_t* __restrict__ t_base,
            int32_t n_sft, fmap_grid g, const float2* __restrict__ wtab, int32_t n_tab,
            const int64_t* __restrict__ ax,
            const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
            const Coef* __restrict__ coef, int32_t shared_antenna, const float* __restrict__ fafb,
            int32_t n_templates, float* __restrict__ map, Partial* __restrict__ parts,
            int64_t stride) {
  constexpr int NCOL = 4 * TC;
  constexpr int LD = NCOL + 4;
  __shared__ __align__(16) float sx[kKC][LD];
  __shared__ int32_t srel[kKC];
  __shared__ Partial scratch[kExpCells / 32];
  __shared__ int32_t s_jmax;
  const int64_t tile = blockIdx.x;
  const int32_t nblk = (g.n_tau + kExpCells - 1) / kExpCells;
  const int32_t m = (int32_t)(tile / nblk);
  const int32_t nn = (int32_t)(tile - (int64_t)m * nblk) * kExpCells + threadIdx.x;
  const bool in_grid = nn < g.n_tau;
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const int64_t cell = (int64_t)m * g.n_tau + (in_grid ? nn : 0);
  const int32_t tq0 = blockIdx.y * TC;
  const int32_t i0 = i0tab[m];
  const int32_t jc = in_grid ? jend[cell] : i0;
  if (threadIdx.x == 0) s_jmax = i0;
  __syncthreads();
  const int32_t jw = __reduce_max_sync(0xffffffffu, jc);
  if ((threadIdx.x & 31) == 0) atomicMax(&s_jmax, jw);
  __syncthreads();
  const int32_t jmax = s_jmax;
  int32_t t0rel = 0;
  if (jmax > i0) t0rel = (int32_t)(grid_t0(g, ax, m) - *t_base);
  const double tau = (double)grid_tau(g, ax, in_grid ? nn : 0);
  const float c2 = (float)(-1.4426950408889634 / tau);
  const double su64 = TAB ? tab_scale(n_tab, exp_cut8_of(g), grid_tau(g, ax, in_grid ? nn : 0)) : 0.0;
  const float su = (float)su64;
  Acc acc[NCOL];
#pragma unroll
  for (int q = 0; q < NCOL; ++q) acc[q] = Acc(0);
  for (int32_t k0 = i0; k0 < jmax; k0 += kKC) {
    __syncthreads();
    for (int e = threadIdx.x; e < NCOL * kKC; e += kExpCells) {
      const int col = e / kKC, kk = e - col * kKC;
      const int32_t a = k0 + kk;
      const int32_t tq = tq0 + (col >> 2);
      float v = 0.0f;
      if (a < jmax && tq < n_templates) v = fafb[((int64_t)tq * 4 + (col & 3)) * n_sft + a];
      sx[kk][col] = v;
    }
    if (threadIdx.x < kKC) {
      const int32_t a = k0 + threadIdx.x;
      srel[threadIdx.x] = a < jmax ? rel_t[a] : 0;
    }
    __syncthreads();
    const int kend = min(kKC, jmax - k0);
    for (int kk = 0; kk < kend; ++kk) {
      const int32_t d = srel[kk] - t0rel;
      Acc w;
      if constexpr (TAB) {
        if constexpr (std::is_same<Acc, double>::value)
          w = (k0 + kk < jc) ? tab_weight64((double)d * su64, wtab, n_tab) : 0.0;
        else
          w = (k0 + kk < jc) ? tab_weight((float)d * su, wtab, n_tab) : 0.0f;
      } else if constexpr (std::is_same<Acc, double>::value) {
        w = (k0 + kk < jc) ? exp(-(double)d / tau) : 0.0;
      } else {
        w = (k0 + kk < jc) ? exp2f((float)d * c2) : 0.0f;
      }
      const float4* row = reinterpret_cast<const float4*>(&sx[kk][0]);
#pragma unroll
      for (int q = 0; q < NCOL / 4; ++q) {
        const float4 v = row[q];
        acc[4 * q + 0] += w * (Acc)v.x;
        acc[4 * q + 1] += w * (Acc)v.y;
        acc[4 * q + 2] += w * (Acc)v.z;
        acc[4 * q + 3] += w * (Acc)v.w;
      }
    }
  }
  const Coef cf0 = coef[cell];
#pragma unroll
  for (int q = 0; q < TC; ++q) {
    const int32_t tq = tq0 + q;
    if (tq >= n_templates) break;
    const Coef cf = shared_antenna ? cf0 : coef[(int64_t)tq * cells + cell];
    const float v = two_f(cf, (float)acc[4 * q], (float)acc[4 * q + 1], (float)acc[4 * q + 2],
                          (float)acc[4 * q + 3]);
    const bool ok = in_grid && cf.valid == 1.0f;
    if (map && in_grid && cf.valid != 2.0f) map[(int64_t)tq * cells + cell] = ok ? v : 0.0f;
    Partial pt = partial_empty();
    partial_add(pt, v, (int32_t)cell, ok);
    pt = partial_block_reduce<kExpCells / 32>(pt, scratch);
    if (threadIdx.x == 0) parts[(int64_t)tq * stride + tile] = pt;
  }
}

cudaError_t launch_exp_plain(fmap_plan_s* p, const fmap_atoms* a, float* d_2F, cudaStream_t s,
                             int64_t* tiles_used) {
  const fmap_grid& g = p->grid;
  const int64_t tiles = exp_tiles(g);
  *tiles_used = tiles;
  p->tiles = TileGeom{0, 1, kExpCells, g.n_t0, (g.n_tau + kExpCells - 1) / kExpCells};
  if (tiles == 0 || p->n_templates == 0) return cudaSuccess;
  const bool tab = g.window == FMAP_TABLE;
  auto run = [&](auto kern, int tc) {
    dim3 grid((unsigned)tiles, (unsigned)((p->n_templates + tc - 1) / tc));
    kern<<<grid, kExpCells, 0, s>>>(p->ws.rel_t, p->ws.t_base, p->n_sft, g, p->ws.wtab, p->n_tab,
                                    plan_axes(p), p->ws.i0, p->ws.jend, p->ws.coef, a->shared_antenna,
                                    a->fafb, p->n_templates, d_2F, p->ws.partials, p->part_stride);
  };
  if (p->precision == FMAP_FP64) {
    if (tab) run(k_exp_plain<double, 8, true>, 8); else run(k_exp_plain<double, 8, false>, 8);
  } else {
    if (tab) run(k_exp_plain<float, 16, true>, 16); else run(k_exp_plain<float, 16, false>, 16);
  }
  p->launches += 1;
  return cudaGetLastError();
}


// ---- persistent multi-instance dispatcher (uneven batches) ----
__global__ void __launch_bounds__(256) kb_exp_perm(const BItem* __restrict__ items, BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    const int32_t n_x = it.perm_x ? it.T : 0;
    const int64_t total = exp_copy_entries(it.n_sft, it.lanes, it.n_ant, n_x, it.g.n_tau);
    const int64_t e0 = k * kPermPerUnit;
    exp_perm_body(it.rel_t, it.n_sft, it.lanes, it.antenna, it.n_ant, it.fafb, n_x, it.perm_ant, it.perm_x,
                  it.perm_gap, it.g, it.ax, it.tauc, e0 + threadIdx.x, min(total, e0 + kPermPerUnit), 256);
  });
}
// (the register budget of 3 blocks of 256 threads per SM, for any width)
template <int NT>
__global__ void __launch_bounds__(NT, 768 / NT) kb_exp_ant(const BItem* __restrict__ items,
                                                        BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    exp_antenna_body<NT>(it.rel_t, it.t_base, it.n_sft, it.g, it.perm_ant, it.tauc, it.ax, it.i0,
                         it.jend, it.coef, it.flag_bits,
                         make_uint3((unsigned)(k % it.g.n_tau), (unsigned)(k / it.g.n_tau), 0),
                         dim3((unsigned)it.g.n_tau, (unsigned)it.n_ant));
  });
}
const void* batch_kernel_exp(int phase, int lanes) {
  if (phase == BP_EXP_PERM) return (const void*)kb_exp_perm;
  if (phase != BP_EXP_ANT) return nullptr;
  return lanes == 64 ? (const void*)kb_exp_ant<64>
                     : lanes == 128 ? (const void*)kb_exp_ant<128> : (const void*)kb_exp_ant<256>;
}
size_t exp_antenna_smem(int32_t n_sft) { return sizeof(float2) * 3 * ((size_t)n_sft + 1); }
bool exp_antenna_fits(int32_t n_sft) { return n_sft <= kAntennaSmemMaxSft; }

}  // namespace fmap
