// Rectangular-window F-map (Eq. winrect).
//
// FMAP_FP64: prefix sums over SFTs in FP64, then O(1) differencing per cell.
//   The antenna rows keep FP64 prefixes (A, B, C and D = AB - C^2 in FP64,
//   once per cell).  The data rows keep each FP64 prefix as an unevaluated
//   float pair hi + lo; a window sum is (hi_j - hi_i) + (lo_j - lo_i), whose
//   rounding error is relative to the window sum itself and not to the
//   (possibly much larger) prefix.
// FMAP_FP32: the paper's rectangular kernel (Sec. 3): one thread per t0 row
//   adds atom after atom to FP32 running sums as tau grows.
#include <math.h>

#include "fmap_batch.cuh"
#include "fmap_device.cuh"

namespace fmap {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr int kCellThreads = 256;

struct __align__(32) D4 {
  double x, y, z, w;
};

int64_t rect_tiles(const fmap_grid& g) {
  return (int64_t)g.n_t0 * ((g.n_tau + kCellThreads - 1) / kCellThreads);
}

// Exclusive block scan of NC doubles per thread (sums of each thread's
// chunk); returns the thread's exclusive prefix in `excl` and the block total
// in `total`.
template <int NC>
__device__ __forceinline__ void block_exscan(const double (&v)[NC], double (&excl)[NC],
                                             double (&total)[NC], double (*sh)[kScanThreads]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int c = 0; c < NC; ++c) sh[c][tid] = v[c];
  __syncthreads();
  // Hillis-Steele inclusive scan in shared memory (log2(256) = 8 steps).
  for (int off = 1; off < kScanThreads; off <<= 1) {
    double add[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) add[c] = tid >= off ? sh[c][tid - off] : 0.0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c) sh[c][tid] += add[c];
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    excl[c] = sh[c][tid] - v[c];
    total[c] = sh[c][kScanThreads - 1];
  }
  __syncthreads();
}

// Prefix of the data rows of one template: px[t][i] = (hi[4], lo[4]) of
// sum_{a < i} x_a for i = 0..N.
__device__ __forceinline__ void rect_scan_data_body(const float* __restrict__ fafb, int32_t n, float4* __restrict__ px,
    const uint3 bid, const dim3 gdim) {
  __shared__ float tile[4][kScanTile];
  __shared__ double sh[4][kScanThreads];
  const int64_t tm = bid.x;
  const float* x = fafb + tm * 4 * (int64_t)n;
  float4* out = px + tm * 2 * (int64_t)(n + 1);
  const int tid = threadIdx.x;
  double carry[4] = {0.0, 0.0, 0.0, 0.0};
  if (tid == 0) {
    out[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    out[1] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int64_t base = 0; base < n; base += kScanTile) {
    for (int k = tid; k < kScanTile; k += kScanThreads) {
      const int64_t a = base + k;
#pragma unroll
      for (int c = 0; c < 4; ++c) tile[c][k] = a < n ? x[c * (int64_t)n + a] : 0.0f;
    }
    __syncthreads();
    double loc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int e = 0; e < kScanPer; ++e)
#pragma unroll
      for (int c = 0; c < 4; ++c) loc[c] += (double)tile[c][tid * kScanPer + e];
    double ex[4], tot[4];
    block_exscan<4>(loc, ex, tot, sh);
    double run[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) run[c] = carry[c] + ex[c];
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
      const int64_t a = base + tid * kScanPer + e;
      float hi[4], lo[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        run[c] += (double)tile[c][tid * kScanPer + e];
        hi[c] = (float)run[c];
        lo[c] = (float)(run[c] - (double)hi[c]);
      }
      if (a < n) {
        out[2 * (a + 1)] = make_float4(hi[0], hi[1], hi[2], hi[3]);
        out[2 * (a + 1) + 1] = make_float4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) carry[c] += tot[c];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads)
k_rect_scan_data(const float* __restrict__ fafb, int32_t n, float4* __restrict__ px) {
  rect_scan_data_body(fafb, n, px, blockIdx, gridDim);
}

// FP64 prefix of the antenna rows: pa[ta][i] = (sum a2, sum b2, sum ab, 0).
__device__ __forceinline__ void rect_scan_antenna_body(const float* __restrict__ antenna, int32_t n, D4* __restrict__ pa,
    const uint3 bid, const dim3 gdim) {
  __shared__ float tile[3][kScanTile];
  __shared__ double sh[3][kScanThreads];
  const int64_t ta = bid.x;
  const float* x = antenna + ta * 3 * (int64_t)n;
  D4* out = pa + ta * (int64_t)(n + 1);
  const int tid = threadIdx.x;
  double carry[3] = {0.0, 0.0, 0.0};
  if (tid == 0) out[0] = D4{0.0, 0.0, 0.0, 0.0};
  for (int64_t base = 0; base < n; base += kScanTile) {
    for (int k = tid; k < kScanTile; k += kScanThreads) {
      const int64_t a = base + k;
#pragma unroll
      for (int c = 0; c < 3; ++c) tile[c][k] = a < n ? x[c * (int64_t)n + a] : 0.0f;
    }
    __syncthreads();
    double loc[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int e = 0; e < kScanPer; ++e)
#pragma unroll
      for (int c = 0; c < 3; ++c) loc[c] += (double)tile[c][tid * kScanPer + e];
    double ex[3], tot[3];
    block_exscan<3>(loc, ex, tot, sh);
    double run[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) run[c] = carry[c] + ex[c];
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
      const int64_t a = base + tid * kScanPer + e;
#pragma unroll
      for (int c = 0; c < 3; ++c) run[c] += (double)tile[c][tid * kScanPer + e];
      if (a < n) out[a + 1] = D4{run[0], run[1], run[2], 0.0};
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) carry[c] += tot[c];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads)
k_rect_scan_antenna(const float* __restrict__ antenna, int32_t n, D4* __restrict__ pa) {
  rect_scan_antenna_body(antenna, n, pa, blockIdx, gridDim);
}

// Per-cell coefficients (shared by the templates of one antenna set) from the
// FP64 antenna prefixes: A, B, C, D = AB - C^2 in FP64.
__device__ __forceinline__ void rect_coef_body(const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
                            const D4* __restrict__ pa, int32_t n_sft, int32_t n_t0, int32_t n_tau,
                            int32_t n_ant, Coef* __restrict__ coef,
    const uint3 bid, const dim3 gdim) {
  const int64_t cells = (int64_t)n_t0 * n_tau;
  const int64_t total = cells * n_ant;
  const int64_t np1 = (int64_t)n_sft + 1;
  for (int64_t e = bid.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gdim.x * blockDim.x) {
    const int64_t ta = e / cells, cell = e - ta * cells;
    const int32_t i0 = i0tab[cell / n_tau], j = jend[cell];
    const D4 pj = pa[ta * np1 + j], pi = pa[ta * np1 + i0];
    coef[e] = make_coef(pj.x - pi.x, pj.y - pi.y, pj.z - pi.z, j - i0);
  }
}

__global__ void k_rect_coef(const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
                            const D4* __restrict__ pa, int32_t n_sft, int32_t n_t0, int32_t n_tau,
                            int32_t n_ant, Coef* __restrict__ coef) {
  rect_coef_body(i0tab, jend, pa, n_sft, n_t0, n_tau, n_ant, coef, blockIdx, gridDim);
}

// One thread per cell (m, n); the block covers 256 consecutive n of one row
// and loops over the templates.  Per template: two float-pair gathers,
// compensated differences, 2F, map store and one block partial.
// Ill-conditioned cells (valid == 2) are left to the FP64 fix-up.
__device__ __forceinline__ void rect_cells_body(const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
             const Coef* __restrict__ coef, const float4* __restrict__ px, int32_t n_sft,
             int32_t n_t0, int32_t n_tau, int32_t n_templates, int32_t shared_antenna,
             float* __restrict__ map, Partial* __restrict__ parts, int64_t stride,
    const uint3 bid, const dim3 gdim) {
  __shared__ Partial scratch[kCellThreads / 32];
  const int64_t tile = bid.x;
  const int32_t nblk = (n_tau + kCellThreads - 1) / kCellThreads;
  const int32_t m = (int32_t)(tile / nblk);
  const int32_t nn = (int32_t)(tile - (int64_t)m * nblk) * kCellThreads + threadIdx.x;
  const bool in_grid = nn < n_tau;
  const int64_t cells = (int64_t)n_t0 * n_tau;
  const int64_t cell = (int64_t)m * n_tau + (in_grid ? nn : 0);
  const int32_t i0 = i0tab[m];
  const int32_t j = in_grid ? jend[cell] : i0;
  const int64_t np1 = (int64_t)n_sft + 1;
  Coef cf = coef[cell];
  for (int32_t tm = 0; tm < n_templates; ++tm) {
    if (!shared_antenna) cf = coef[(int64_t)tm * cells + cell];
    const float4* pt = px + (int64_t)tm * 2 * np1;
    const float4 hj = pt[2 * (int64_t)j], lj = pt[2 * (int64_t)j + 1];
    const float4 hi = pt[2 * (int64_t)i0], li = pt[2 * (int64_t)i0 + 1];
    const float fa_re = (hj.x - hi.x) + (lj.x - li.x);
    const float fa_im = (hj.y - hi.y) + (lj.y - li.y);
    const float fb_re = (hj.z - hi.z) + (lj.z - li.z);
    const float fb_im = (hj.w - hi.w) + (lj.w - li.w);
    const float v = two_f(cf, fa_re, fa_im, fb_re, fb_im);
    const bool ok = in_grid && cf.valid == 1.0f;
    if (map && in_grid && cf.valid != 2.0f) map[(int64_t)tm * cells + cell] = ok ? v : 0.0f;
    Partial p = partial_empty();
    partial_add(p, v, (int32_t)cell, ok);
    p = partial_block_reduce<kCellThreads / 32>(p, scratch);
    if (threadIdx.x == 0) parts[(int64_t)tm * stride + tile] = p;
  }
}

__global__ void __launch_bounds__(kCellThreads)
k_rect_cells(const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
             const Coef* __restrict__ coef, const float4* __restrict__ px, int32_t n_sft,
             int32_t n_t0, int32_t n_tau, int32_t n_templates, int32_t shared_antenna,
             float* __restrict__ map, Partial* __restrict__ parts, int64_t stride) {
  rect_cells_body(i0tab, jend, coef, px, n_sft, n_t0, n_tau, n_templates, shared_antenna, map, parts, stride, blockIdx, gridDim);
}

// The paper's rectangular kernel (Sec. 3) for the data rows: one thread per
// (template, t0 row), FP32 running sums of Fa, Fb extended as tau grows; the
// antenna part comes from the FP64 coefficients.
constexpr int kRowThreads = 128;

__global__ void __launch_bounds__(kRowThreads)
k_rect_rows_fp32(const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
                 const Coef* __restrict__ coef, const float* __restrict__ fafb, int32_t n_sft,
                 int32_t n_t0, int32_t n_tau, int32_t shared_antenna, float* __restrict__ map,
                 Partial* __restrict__ parts, int64_t stride) {
  __shared__ Partial scratch[kRowThreads / 32];
  const int32_t m = blockIdx.x * kRowThreads + threadIdx.x;
  const int64_t tm = blockIdx.y;
  const int64_t cells = (int64_t)n_t0 * n_tau;
  const float* x = fafb + tm * 4 * (int64_t)n_sft;
  const Coef* cp = coef + (shared_antenna ? 0 : tm * cells);
  Partial acc = partial_empty();
  if (m < n_t0) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int32_t a = i0tab[m];
    for (int32_t nn = 0; nn < n_tau; ++nn) {
      const int64_t cell = (int64_t)m * n_tau + nn;
      const int32_t j = jend[cell];
      for (; a < j; ++a) {
        s0 += x[a];
        s1 += x[n_sft + a];
        s2 += x[2 * (int64_t)n_sft + a];
        s3 += x[3 * (int64_t)n_sft + a];
      }
      const Coef cf = cp[cell];
      const float v = two_f(cf, s0, s1, s2, s3);
      const bool ok = cf.valid == 1.0f;
      if (map && cf.valid != 2.0f) map[tm * cells + cell] = ok ? v : 0.0f;
      partial_add(acc, v, (int32_t)cell, ok);
    }
  }
  acc = partial_block_reduce<kRowThreads / 32>(acc, scratch);
  if (threadIdx.x == 0) parts[tm * stride + blockIdx.x] = acc;
}

cudaError_t launch_rect_coef(fmap_plan_s* p, const fmap_atoms* a, cudaStream_t s) {
  const fmap_grid& g = p->grid;
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  if (cells == 0) return cudaSuccess;
  const int n_ant = a->shared_antenna ? 1 : p->n_templates;
  if (n_ant == 0) return cudaSuccess;
  if (p->n_sft > 0) {
    k_rect_scan_antenna<<<n_ant, kScanThreads, 0, s>>>(a->antenna, p->n_sft, (D4*)p->ws.pa);
  } else {
    cudaMemsetAsync(p->ws.pa, 0, sizeof(D4) * n_ant, s);
  }
  const int64_t total = cells * n_ant;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)p->n_sm * 16);
  k_rect_coef<<<blocks, 256, 0, s>>>(p->ws.i0, p->ws.jend, (const D4*)p->ws.pa, p->n_sft, g.n_t0,
                                     g.n_tau, n_ant, p->ws.coef);
  p->launches += (p->n_sft > 0) ? 2 : 1;
  return cudaGetLastError();
}

cudaError_t launch_rect(fmap_plan_s* p, const fmap_atoms* a, float* d_2F, cudaStream_t s,
                        int64_t* tiles_used, cudaEvent_t mark) {
  const fmap_grid& g = p->grid;
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  *tiles_used = 0;
  if (cells == 0 || p->n_templates == 0) return cudaSuccess;
  if (p->precision == FMAP_FP32) {
    if (mark) cudaEventRecord(mark, s);
    dim3 grid((unsigned)((g.n_t0 + kRowThreads - 1) / kRowThreads), (unsigned)p->n_templates);
    *tiles_used = grid.x;
    k_rect_rows_fp32<<<grid, kRowThreads, 0, s>>>(p->ws.i0, p->ws.jend, p->ws.coef, a->fafb,
                                                  p->n_sft, g.n_t0, g.n_tau, a->shared_antenna,
                                                  d_2F, p->ws.partials, p->part_stride);
    p->launches += 1;
    return cudaGetLastError();
  }
  if (p->n_sft > 0) {
    k_rect_scan_data<<<p->n_templates, kScanThreads, 0, s>>>(a->fafb, p->n_sft, p->ws.px);
    p->launches += 1;
  } else {
    cudaMemsetAsync(p->ws.px, 0, 2 * sizeof(float4) * p->n_templates, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (mark) cudaEventRecord(mark, s);
  const int64_t tiles = rect_tiles(g);
  *tiles_used = tiles;
  k_rect_cells<<<(unsigned)tiles, kCellThreads, 0, s>>>(
      p->ws.i0, p->ws.jend, p->ws.coef, p->ws.px, p->n_sft, g.n_t0, g.n_tau, p->n_templates,
      a->shared_antenna, d_2F, p->ws.partials, p->part_stride);
  p->launches += 1;
  return cudaGetLastError();
}


// ---- persistent multi-instance dispatchers (uneven batches) ----
__global__ void __launch_bounds__(kScanThreads) kb_rect_ant(const BItem* __restrict__ items,
                                                            BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    rect_scan_antenna_body(it.antenna, it.n_sft, (D4*)it.pa, make_uint3((unsigned)k, 0, 0),
                           dim3((unsigned)it.n_ant));
  });
}
__global__ void __launch_bounds__(256) kb_rect_coef(const BItem* __restrict__ items, BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    rect_coef_body(it.i0, it.jend, (const D4*)it.pa, it.n_sft, it.g.n_t0, it.g.n_tau, it.n_ant,
                   it.coef, make_uint3((unsigned)k, 0, 0),
                   dim3((unsigned)((it.cells * it.n_ant + 255) / 256)));
  });
}
__global__ void __launch_bounds__(kScanThreads) kb_rect_data(const BItem* __restrict__ items,
                                                             BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    rect_scan_data_body(it.fafb, it.n_sft, it.px, make_uint3((unsigned)k, 0, 0),
                        dim3((unsigned)it.T));
  });
}
__global__ void __launch_bounds__(kCellThreads) kb_rect_cells(const BItem* __restrict__ items,
                                                              BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    rect_cells_body(it.i0, it.jend, it.coef, it.px, it.n_sft, it.g.n_t0, it.g.n_tau, it.T,
                    it.shared, it.map, it.partials, it.part_stride, make_uint3((unsigned)k, 0, 0),
                    dim3((unsigned)it.tiles_used));
  });
}
const void* batch_kernel_rect(int phase) {
  switch (phase) {
    case BP_RECT_ANT: return (const void*)kb_rect_ant;
    case BP_RECT_COEF: return (const void*)kb_rect_coef;
    case BP_RECT_DATA: return (const void*)kb_rect_data;
    case BP_RECT_CELLS: return (const void*)kb_rect_cells;
  }
  return nullptr;
}

}  // namespace fmap
