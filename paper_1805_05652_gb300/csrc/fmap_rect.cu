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

constexpr int kTileRows = 4;    // t0 rows of a warp tile of the cells kernel
constexpr int kTileCols = 64;   // tau columns of a warp tile

// Warp tiles of the cells kernel: one partial per (template, tile).
int64_t rect_tiles(const fmap_grid& g) {
  return (int64_t)((g.n_t0 + kTileRows - 1) / kTileRows) *
         ((g.n_tau + kTileCols - 1) / kTileCols);
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

// Cells, one warp per unit of (warp tile, template chunk).
//
// A warp tile is kTileRows t0 rows x kTileCols tau columns; lane l holds the
// cells (m0 + r, n0 + l + 32 q), r < kTileRows, q < 2, with their
// coefficients in registers, and runs over the kWarpTemplates templates of
// its chunk.  For each template the prefix entries the tile needs (the rows'
// window starts i0 and the contiguous range of window ends) are copied to
// the warp's shared memory with cp.async one template ahead, then rebased to
// the tile's first start b = i0(m0): Q[k] = (hi_k - hi_b) + (lo_k - lo_b).
// A window sum is Q[j] - Q[i0]; its rounding error is relative to the sums
// over [b, j) and [b, i0), i.e. to the window plus the few atoms between the
// tile's rows, so the staged form is used only when those rows span at most
// kMaxRowSpread atoms (and the entries fit the stage); other tiles difference
// the float pairs straight from global memory.
//
// Per template the warp stores the 2F of its cells (coalesced 128-byte
// rows) and writes one partial: the warp maximum by an integer max over the
// 2F bit patterns (2F >= 0), then the lanes' exp-sums rescaled to it, the
// lowest cell index attaining it, and the valid count.  Invalid and
// ill-conditioned cells carry k1 = NaN, so their 2F is NaN: fmaxf drops it
// from the maximum and the exp-sum, it never equals the maximum, and the map
// gets 0 (the FP64 fix-up later rewrites the ill-conditioned ones).
constexpr int kLaneCells = kTileRows * (kTileCols / 32);
constexpr int kWarpTemplates = 16;
constexpr int kStageEntries = 192;
constexpr int kMaxRowSpread = 64;
constexpr int kCellWarps = kCellThreads / 32;
constexpr size_t kWarpStageBytes = (size_t)kStageEntries * (32 + 16);

size_t rect_cells_smem() { return kWarpStageBytes * kCellWarps; }

int64_t rect_blocks(const fmap_grid& g, int32_t n_templates) {
  const int64_t units = rect_tiles(g) * ((n_templates + kWarpTemplates - 1) / kWarpTemplates);
  return (units + kCellWarps - 1) / kCellWarps;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;\n" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ void st_stream(float* p, float v) {
  asm volatile("st.global.cs.f32 [%0], %1;\n" ::"l"(p), "f"(v) : "memory");
}

template <bool kShared>
__device__ __forceinline__ void rect_cells_body(const int32_t* __restrict__ i0tab,
    const int32_t* __restrict__ jend, const Coef* __restrict__ coef,
    const float4* __restrict__ px, int32_t n_sft, int32_t n_t0, int32_t n_tau,
    int32_t n_templates, float* __restrict__ map, Partial* __restrict__ parts, int64_t stride,
    int64_t blk, unsigned char* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t n_rg = (n_t0 + kTileRows - 1) / kTileRows;
  const int32_t n_ct = (n_tau + kTileCols - 1) / kTileCols;
  const int32_t n_wc = (n_templates + kWarpTemplates - 1) / kWarpTemplates;
  const int64_t unit = blk * kCellWarps + warp;
  if (n_wc == 0 || unit >= (int64_t)n_rg * n_ct * n_wc) return;
  // Chunks of one tile are neighbours (coefficients shared through L1/L2);
  // tiles run down a column of row groups (nearby prefix ranges in flight).
  const int32_t wc = (int32_t)(unit % n_wc);
  const int64_t wt = unit / n_wc;
  const int32_t ct = (int32_t)(wt / n_rg), rg = (int32_t)(wt - (int64_t)ct * n_rg);
  const int32_t m0 = rg * kTileRows, n0 = ct * kTileCols;
  const int32_t rows = min(kTileRows, n_t0 - m0);
  const int64_t cells = (int64_t)n_t0 * n_tau;
  const int64_t np1 = (int64_t)n_sft + 1;
  const int64_t cell0 = (int64_t)m0 * n_tau + n0 + lane;   // lane's cell in row 0, q = 0
  const int32_t jmin = jend[(int64_t)m0 * n_tau + n0];
  const int32_t jmax = jend[(int64_t)(m0 + rows - 1) * n_tau + min(n0 + kTileCols, n_tau) - 1];
  const int32_t rj = jmax - jmin + 1;
  const bool staged = kTileRows + rj <= kStageEntries &&
                      i0tab[m0 + rows - 1] - i0tab[m0] <= kMaxRowSpread;

  unsigned char* wsm = smem + (size_t)warp * kWarpStageBytes;
  float4* raw = (float4*)wsm;                               // staged: [entry][hi, lo]
  float4* Q = (float4*)(wsm + (size_t)kStageEntries * 32);  // staged: rebased prefixes
  const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(raw);

  const bool col0 = n0 + lane < n_tau, col1 = n0 + lane + 32 < n_tau;
  auto in_grid = [&](int i) { return (i >> 1) < rows && ((i & 1) ? col1 : col0); };
  auto cell_off = [&](int i) { return (int64_t)(i >> 1) * n_tau + 32 * (i & 1); };

  // Staged: the lane's window ends as entries of Q, two 16-bit indices per word.
  uint32_t jp[kLaneCells / 2];
#pragma unroll
  for (int r = 0; r < kTileRows; ++r) {
    uint32_t w = 0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = 2 * r + q;
      const int32_t j = in_grid(i) ? jend[cell0 + cell_off(i)] : jmin;
      w |= (uint32_t)(kTileRows + (j - jmin)) << (16 * q);
    }
    jp[r] = staged ? w : 0u;
  }

  float k1[kLaneCells], be[kLaneCells], k2[kLaneCells];
  int32_t nval = 0;
  auto load_coef = [&](const Coef* __restrict__ cb) {
    int32_t c = 0;
#pragma unroll
    for (int i = 0; i < kLaneCells; ++i) {
      Coef cf{0.0f, 0.0f, 0.0f, 0.0f};
      if (in_grid(i)) cf = cb[cell0 + cell_off(i)];
      const bool ok = cf.valid == 1.0f;
      k1[i] = ok ? cf.k1 : __int_as_float(0x7fc00000);
      be[i] = cf.beta;
      k2[i] = cf.k2;
      c += ok ? 1 : 0;
    }
    nval = (int32_t)__reduce_add_sync(0xffffffffu, (unsigned)c);
  };
  if (kShared) load_coef(coef);

  auto issue = [&](int32_t tm) {
    const float4* pt = px + (int64_t)tm * 2 * np1;
    const int n_chunk = 2 * (kTileRows + rj);
    for (int c = lane; c < n_chunk; c += 32) {
      const int e = c >> 1;
      const int32_t idx = e < kTileRows ? i0tab[m0 + min(e, rows - 1)] : jmin + (e - kTileRows);
      cp_async16(raw_s + (uint32_t)c * 16u, pt + 2 * (int64_t)idx + (c & 1));
    }
    cp_async_commit();
  };

  const int32_t t_begin = wc * kWarpTemplates;
  const int32_t t_end = min(n_templates, t_begin + kWarpTemplates);
  if (staged) issue(t_begin);
  constexpr float kHalfLog2e = 0.72134752044448170368f;   // log2(e) / 2
  for (int32_t tm = t_begin; tm < t_end; ++tm) {
    if (!kShared) load_coef(coef + (int64_t)tm * cells);
    if (staged) {
      cp_async_wait_all();
      __syncwarp();
      const float4 hb = raw[0], lb = raw[1];
      for (int e = lane; e < kTileRows + rj; e += 32) {
        const float4 h = raw[2 * e], l = raw[2 * e + 1];
        Q[e] = make_float4((h.x - hb.x) + (l.x - lb.x), (h.y - hb.y) + (l.y - lb.y),
                           (h.z - hb.z) + (l.z - lb.z), (h.w - hb.w) + (l.w - lb.w));
      }
      __syncwarp();
      if (tm + 1 < t_end) issue(tm + 1);
    } else {
      // Window sums of the lane's cells from the float pairs in global
      // memory, parked in the (unused) stage buffer: raw[i * 32 + lane].
      const float4* pt = px + (int64_t)tm * 2 * np1;
      __syncwarp();
#pragma unroll 1
      for (int i = 0; i < kLaneCells; ++i) {
        const int32_t mr = m0 + min(i >> 1, rows - 1);
        const int32_t i0 = i0tab[mr];
        const int32_t j = in_grid(i) ? jend[cell0 + cell_off(i)] : i0;
        const float4 hi = pt[2 * (int64_t)i0], li = pt[2 * (int64_t)i0 + 1];
        const float4 hj = pt[2 * (int64_t)j], lj = pt[2 * (int64_t)j + 1];
        raw[i * 32 + lane] = make_float4((hj.x - hi.x) + (lj.x - li.x), (hj.y - hi.y) + (lj.y - li.y),
                                         (hj.z - hi.z) + (lj.z - li.z), (hj.w - hi.w) + (lj.w - li.w));
      }
      __syncwarp();
    }
    float v[kLaneCells];
    float mx = -1.0f;
#pragma unroll
    for (int i = 0; i < kLaneCells; ++i) {
      float4 w;
      if (staged) {
        const float4 qi = Q[i >> 1];
        const float4 qj = Q[(jp[i >> 1] >> (16 * (i & 1))) & 0xffffu];
        w = make_float4(qj.x - qi.x, qj.y - qi.y, qj.z - qi.z, qj.w - qi.w);
      } else {
        w = raw[i * 32 + lane];
      }
      const Coef cf{k1[i], be[i], k2[i], 1.0f};
      v[i] = two_f(cf, w.x, w.y, w.z, w.w);
      mx = fmaxf(mx, v[i]);
    }
    if (map) {
      float* mt = map + (int64_t)tm * cells + cell0;
#pragma unroll
      for (int i = 0; i < kLaneCells; ++i)
        if (in_grid(i)) st_stream(mt + cell_off(i), fmaxf(v[i], 0.0f));
    }
    // 2F >= 0, so its bit pattern orders like the value; 0 marks "no valid cell".
    const unsigned mu = __reduce_max_sync(0xffffffffu, mx >= 0.0f ? __float_as_uint(mx) + 1u : 0u);
    if (mu == 0u) {
      if (lane == 0) parts[(int64_t)tm * stride + wt] = partial_empty();
      continue;
    }
    const float M = __uint_as_float(mu - 1u);
    const float mc = -M * kHalfLog2e;
    float s = 0.0f;
    int32_t arg = kNoArg;
#pragma unroll
    for (int i = kLaneCells - 1; i >= 0; --i) {
      s += fmaxf(ex2_approx(fmaf(v[i], kHalfLog2e, mc)), 0.0f);
      if (v[i] == M) arg = (int32_t)(cell0 + cell_off(i));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    arg = (int32_t)__reduce_min_sync(0xffffffffu, (unsigned)arg);
    if (lane == 0) {
      Partial p;
      p.max2F = M;
      p.arg = arg;
      p.sum = s;
      p.nvalid = nval;
      parts[(int64_t)tm * stride + wt] = p;
    }
  }
}

template <bool kShared>
__global__ void __launch_bounds__(kCellThreads, 2)
k_rect_cells(const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
             const Coef* __restrict__ coef, const float4* __restrict__ px, int32_t n_sft,
             int32_t n_t0, int32_t n_tau, int32_t n_templates, float* __restrict__ map,
             Partial* __restrict__ parts, int64_t stride) {
  extern __shared__ __align__(16) unsigned char s_cells[];
  rect_cells_body<kShared>(i0tab, jend, coef, px, n_sft, n_t0, n_tau, n_templates, map, parts,
                           stride, blockIdx.x, s_cells);
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
  *tiles_used = rect_tiles(g);
  const int64_t blocks = rect_blocks(g, p->n_templates);
  if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  const void* kfn = a->shared_antenna ? (const void*)k_rect_cells<true> : (const void*)k_rect_cells<false>;
  e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rect_cells_smem());
  if (e != cudaSuccess) return e;
  if (a->shared_antenna)
    k_rect_cells<true><<<(unsigned)blocks, kCellThreads, rect_cells_smem(), s>>>(
        p->ws.i0, p->ws.jend, p->ws.coef, p->ws.px, p->n_sft, g.n_t0, g.n_tau, p->n_templates,
        d_2F, p->ws.partials, p->part_stride);
  else
    k_rect_cells<false><<<(unsigned)blocks, kCellThreads, rect_cells_smem(), s>>>(
        p->ws.i0, p->ws.jend, p->ws.coef, p->ws.px, p->n_sft, g.n_t0, g.n_tau, p->n_templates,
        d_2F, p->ws.partials, p->part_stride);
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
__global__ void __launch_bounds__(kCellThreads, 2) kb_rect_cells(const BItem* __restrict__ items,
                                                                 BUnits u) {
  extern __shared__ __align__(16) unsigned char s_cells[];
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    if (it.shared)
      rect_cells_body<true>(it.i0, it.jend, it.coef, it.px, it.n_sft, it.g.n_t0, it.g.n_tau,
                            it.T, it.map, it.partials, it.part_stride, k, s_cells);
    else
      rect_cells_body<false>(it.i0, it.jend, it.coef, it.px, it.n_sft, it.g.n_t0, it.g.n_tau,
                             it.T, it.map, it.partials, it.part_stride, k, s_cells);
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
