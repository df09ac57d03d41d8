// Generic window functions (FMAP_TABLE grids).
//
// The paper's kernels take the rectangular and exponential windows; its
// method is the same for any amplitude envelope w of the transient: the atoms
// of a window enter Fa, Fb with the weight w((t - t0) / tau) and A, B, C with
// w^2.  Here w is a table of samples on [0, X], X = exp_cut8 / 8 (linear
// between samples, 0 past X), over the exponential window's support.
//
// The data sums go through the same contraction kernels as the exponential
// window (W generated from the table instead of exp2).  The antenna sums
// have no recurrence for a generic w, so this file sums them directly over
// each window: one block per (t0 row, 128 tau cells, antenna set), each warp
// staging the atoms of its 32 cells' windows in shared memory (up to the
// longest of them, so that a warp never waits for another), every cell
// accumulating its window
// by cascaded (Sum2) summation with exact products (the FP32 weights act as a
// slightly perturbed window, the same for A, B and C; the sums carry about
// twice-working-precision accuracy, enough for D = AB - C^2 up to AB/D = 100).
#include <math.h>

#include "fmap_device.cuh"

namespace fmap {

constexpr int kTabCells = 128;   // tau cells of a block (one t0 row)
constexpr int kTabKC = 64;       // atoms staged per round
constexpr int kTabWarps = kTabCells / 32;

// S += a b in the cascaded form of Ogita, Rump and Oishi's Sum2 with an exact
// product: S.h is the plain FP32 running sum, S.l collects the product's
// FMA error and the TwoSum error of each addition (folded into S.h once, at
// the end, by ff_fold); the result is as accurate as summing in twice the
// working precision.
__device__ __forceinline__ void ff_add_prod(FF& S, float a, float b) {
  const float p = a * b;
  const float pe = fmaf(a, b, -p);
  const float s = S.h + p;
  const float bb = s - S.h;
  const float se = (S.h - (s - bb)) + (p - bb);
  S.l += se + pe;
  S.h = s;
}
__device__ __forceinline__ FF ff_fold(FF S) { return fast_two_sum(S.h, S.l); }

__global__ void __launch_bounds__(kTabCells)
k_table_antenna(const int32_t* __restrict__ rel_t, const int64_t* __restrict__ t_base, int32_t n,
                fmap_grid g, const int64_t* __restrict__ ax, const float2* __restrict__ wtab,
                int32_t n_tab, const float* __restrict__ antenna,
                const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
                Coef* __restrict__ coef, uint32_t* __restrict__ bits) {
  __shared__ float s_t[kTabWarps][kTabKC];
  __shared__ float s_a[kTabWarps][3][kTabKC];
  __shared__ float2 s_tab[kTabMax + 1];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int32_t nblk = (g.n_tau + kTabCells - 1) / kTabCells;
  const int32_t m = (int32_t)(blockIdx.x / nblk);
  const int32_t nn = (int32_t)(blockIdx.x - m * nblk) * kTabCells + tid;
  const int ta = blockIdx.y;
  const bool in_grid = nn < g.n_tau;
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const int64_t cell = (int64_t)m * g.n_tau + (in_grid ? nn : 0);
  for (int k = tid; k <= n_tab; k += kTabCells) s_tab[k] = wtab[k];
  const int32_t i0 = i0tab[m];
  const int32_t jc = in_grid ? jend[cell] : i0;
  __syncthreads();   // the table is staged
  const int32_t jmax = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)jc);   // the warp's
  const int64_t tb = n > 0 ? *t_base : 0;
  const int64_t t0rel = grid_t0(g, ax, m) - tb;
  const float su =
      in_grid ? (float)tab_scale(n_tab, exp_cut8_of(g), grid_tau(g, ax, nn)) : 0.0f;
  const float* ant = antenna + (int64_t)ta * 3 * n;
  FF S[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int32_t k0 = i0; k0 < jmax; k0 += kTabKC) {
    __syncwarp();   // the warp's previous round is read
    for (int e = lane; e < kTabKC; e += 32) {
      const int32_t a = k0 + e;
      const bool in = a < jmax;
      s_t[w][e] = in ? (float)((int64_t)rel_t[a] - t0rel) : 0.0f;
#pragma unroll
      for (int c = 0; c < 3; ++c) s_a[w][c][e] = in ? ant[(int64_t)c * n + a] : 0.0f;
    }
    __syncwarp();
    const int kend = min(kTabKC, jc - k0);   // this cell's atoms in the round
    for (int kk = 0; kk < kend; ++kk) {
      const float wt = tab_weight(s_t[w][kk] * su, s_tab, n_tab);
      const float w2 = wt * wt;
#pragma unroll
      for (int c = 0; c < 3; ++c) ff_add_prod(S[c], w2, s_a[w][c][kk]);
    }
  }
  if (in_grid)
    store_coef(coef, bits, (int64_t)ta * cells + cell,
               make_coef_ff(ff_fold(S[0]), ff_fold(S[1]), ff_fold(S[2]), jc - i0));
}

cudaError_t launch_table_antenna(fmap_plan_s* p, const fmap_atoms* a, cudaStream_t s) {
  const fmap_grid& g = p->grid;
  if ((int64_t)g.n_t0 * g.n_tau == 0) return cudaSuccess;
  const int n_ant = a->shared_antenna ? 1 : p->n_templates;
  const int64_t blocks = (int64_t)g.n_t0 * ((g.n_tau + kTabCells - 1) / kTabCells);
  k_table_antenna<<<dim3((unsigned)blocks, (unsigned)n_ant), kTabCells, 0, s>>>(
      p->ws.rel_t, p->ws.t_base, p->n_sft, g, plan_axes(p), p->ws.wtab, p->n_tab, a->antenna,
      p->ws.i0, p->ws.jend, p->ws.coef, p->ws.flag_bits);
  p->launches += 1;
  return cudaGetLastError();
}

}  // namespace fmap
