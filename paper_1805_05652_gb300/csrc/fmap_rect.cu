// Rectangular-window F-map (Eq. winrect).
//
// FMAP_FP64: prefix sums over SFTs in FP64, then O(1) differencing per cell.
//   Every FP64 prefix is kept as an unevaluated float pair hi + lo; a window
//   sum is (hi_j - hi_i) + (lo_j - lo_i), whose rounding error is relative
//   to the window sum itself and not to the (possibly much larger) prefix.
//   The antenna sums A, B, C are differenced in float-float (~2^-44 of the
//   prefix) and D = AB - C^2 formed from exact FMA products; cells with
//   AB > 100 D go to the fix-up.  (GB300 runs FP64 at 1/64 of the FP32
//   rate, so the per-cell work stays off the FP64 pipe.)
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

// Antenna prefix entry: (sum a2, sum b2, sum ab, 0) as float pairs.
struct __align__(32) P4 {
  float4 hi, lo;
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

// FP64 prefix of the antenna rows, stored as float pairs: pa[ta][i] =
// (sum a2, sum b2, sum ab, 0) over a < i.
__device__ __forceinline__ void rect_scan_antenna_body(const float* __restrict__ antenna, int32_t n, P4* __restrict__ pa,
    const uint3 bid, const dim3 gdim) {
  __shared__ float tile[3][kScanTile];
  __shared__ double sh[3][kScanThreads];
  const int64_t ta = bid.x;
  const float* x = antenna + ta * 3 * (int64_t)n;
  P4* out = pa + ta * (int64_t)(n + 1);
  const int tid = threadIdx.x;
  double carry[3] = {0.0, 0.0, 0.0};
  if (tid == 0) out[0] = P4{make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
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
      if (a < n) {
        float hi[3], lo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          hi[c] = (float)run[c];
          lo[c] = (float)(run[c] - (double)hi[c]);
        }
        out[a + 1] = P4{make_float4(hi[0], hi[1], hi[2], 0.f), make_float4(lo[0], lo[1], lo[2], 0.f)};
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) carry[c] += tot[c];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads)
k_rect_scan_antenna(const float* __restrict__ antenna, int32_t n, P4* __restrict__ pa) {
  rect_scan_antenna_body(antenna, n, pa, blockIdx, gridDim);
}

// Per-cell coefficients (shared by the templates of one antenna set) from the
// antenna prefixes: A, B, C as float-float differences, D = AB - C^2 from
// exact FMA products.
__device__ __forceinline__ Coef rect_cell_coef(const P4* __restrict__ pa, int64_t e_i0,
                                               int64_t e_j, int32_t count) {
  const P4 pj = pa[e_j], pi = pa[e_i0];
  const FF A = ff_sub(FF{pj.hi.x, pj.lo.x}, FF{pi.hi.x, pi.lo.x});
  const FF B = ff_sub(FF{pj.hi.y, pj.lo.y}, FF{pi.hi.y, pi.lo.y});
  const FF C = ff_sub(FF{pj.hi.z, pj.lo.z}, FF{pi.hi.z, pi.lo.z});
  return make_coef_ff(A, B, C, count);
}

__device__ __forceinline__ void rect_coef_body(const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
                            const P4* __restrict__ pa, int32_t n_sft, int32_t n_t0, int32_t n_tau,
                            int32_t n_ant, Coef* __restrict__ coef, uint32_t* __restrict__ bits,
    const uint3 bid, const dim3 gdim) {
  const int64_t cells = (int64_t)n_t0 * n_tau;
  const int64_t total = cells * n_ant;
  const int64_t np1 = (int64_t)n_sft + 1;
  const int64_t step = (int64_t)gdim.x * blockDim.x;
  const int64_t e0 = bid.x * (int64_t)blockDim.x + threadIdx.x;
  if (total <= 0xffffffffll) {
    // 32-bit index arithmetic (the usual case)
    const uint32_t ucells = (uint32_t)cells, utau = (uint32_t)n_tau;
    for (int64_t e = e0; e < total; e += step) {
      const uint32_t ue = (uint32_t)e;
      const uint32_t ta = ue / ucells, cell = ue - ta * ucells;
      const int32_t i0 = i0tab[cell / utau], j = jend[cell];
      store_coef(coef, bits, e, rect_cell_coef(pa, ta * np1 + i0, ta * np1 + j, j - i0));
    }
    return;
  }
  for (int64_t e = e0; e < total; e += step) {
    const int64_t ta = e / cells, cell = e - ta * cells;
    const int32_t i0 = i0tab[cell / n_tau], j = jend[cell];
    store_coef(coef, bits, e, rect_cell_coef(pa, ta * np1 + i0, ta * np1 + j, j - i0));
  }
}

__global__ void k_rect_coef(const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
                            const P4* __restrict__ pa, int32_t n_sft, int32_t n_t0, int32_t n_tau,
                            int32_t n_ant, Coef* __restrict__ coef, uint32_t* __restrict__ bits) {
  rect_coef_body(i0tab, jend, pa, n_sft, n_t0, n_tau, n_ant, coef, bits, blockIdx, gridDim);
}

// Cells.  The unit of work is a warp tile of kTileRows t0 rows x kTileCols
// tau columns and one template; lane l holds the cells (m0 + r, n0 + l +
// 32 q), r < kTileRows, q < 2, with their coefficients in registers, and
// each (template, warp tile) gets one partial.
//
// Two warp tiles stacked in rows form a group of kGroupRows rows that share
// one rebase.  A block holds 4 / tl groups and tl template lanes per warp
// tile (tl = 4, 2 or 1 by the template count, so small batches still fill
// the block), and runs a chunk of kBlockTemplates templates in stages of
// 2 tl templates.  A stage has kSlots (group, template) slots, slot w owned
// by warp w; for each, the prefix entries of the group's row starts and of
// its contiguous range of window ends are fetched with two bulk copies (TMA,
// completing on the slot's mbarrier) one stage ahead, then rebased by the
// owner warp to the group's first start b: Q[k] = (hi_k - hi_b) +
// (lo_k - lo_b), into one of two Q buffers; the two warps of a tile pair
// that read each other's slots meet at a named barrier.  A window sum is Q[j] - Q[i0], one FP32 difference whose
// rounding error is relative to the sums over [b, j) and [b, i0): the
// window plus the few atoms between the group's rows.  Blocks whose groups
// span more than kMaxRowSpread atoms between rows, or whose entries do not
// fit a slot, difference the float pairs straight from global memory.
//
// Per template a warp stores the 2F of its cells (128-byte row pieces,
// streaming stores) and writes one partial: the warp maximum by an integer
// max over the 2F bit patterns (2F >= 0), the lanes' exp-sums rescaled to
// it, the lowest cell index attaining it and the valid count.  Invalid and
// ill-conditioned cells carry k1 = -inf (|Fa|^2 is kept >= 1e-30 so the
// product is -inf, never NaN): the maximum ignores them, their exp-term is
// 0, they never equal the maximum, and the map gets 0 (the fix-up later
// rewrites the ill-conditioned ones).  The quadratic form runs on packed
// f32x2 arithmetic (re, im pairs).
constexpr int kLaneCells = kTileRows * (kTileCols / 32);
constexpr int kCellWarps = kCellThreads / 32;
constexpr int kGroupRows = 2 * kTileRows;
constexpr int kSlots = 8;
constexpr int kRowCap = 40;            // row-start entries of a slot
constexpr int kJCap = 152;             // window-end entries of a slot
constexpr int kSlotEntries = kRowCap + kJCap;
// Atoms between a group's first and last row start: a window sum's rounding
// error grows with the atoms between the group's base and the window (its
// own rows' starts lie up to this many atoms past the base).  At 32 a
// numpy emulation of this kernel's roundings found 1.1e-5 relative 2F on
// 4-atom windows of A B / D ~ 40 at t0 steps of ~2 SFTs (over the 1e-5
// bar); at 8, 2.9e-6 worst over the same instances.
constexpr int kMaxRowSpread = 8;
constexpr int kBlockTemplates = 128;
constexpr size_t kRawBytes = (size_t)kSlots * kSlotEntries * 32;
constexpr size_t kQBytes = (size_t)kSlots * kSlotEntries * 16;
static_assert((size_t)kCellWarps * kLaneCells * 32 * 16 <= kRawBytes,
              "global-path window sums must fit in the stage buffer");

// Template lanes per warp tile.
__host__ __device__ __forceinline__ int rect_tlanes(int32_t n_templates) {
  return n_templates >= 4 ? 4 : (n_templates >= 2 ? 2 : 1);
}

static size_t rect_cmaj_smem() { return kRawBytes + 2 * kQBytes; }

static int64_t rect_cmaj_blocks(const fmap_grid& g, int32_t n_templates) {
  const int32_t brows = kGroupRows * (4 / rect_tlanes(n_templates));
  return (int64_t)((g.n_t0 + brows - 1) / brows) * ((g.n_tau + kTileCols - 1) / kTileCols) *
         ((n_templates + kBlockTemplates - 1) / kBlockTemplates);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;\n" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ void st_stream(float* p, float v) {
  asm volatile("st.global.cs.f32 [%0], %1;\n" ::"l"(p), "f"(v) : "memory");
}
// f32x2 pairs: .x in the low half.
__device__ __forceinline__ void lds_pairs(uint32_t a, uint64_t& xy, uint64_t& zw) {
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];\n" : "=l"(xy), "=l"(zw) : "r"(a));
}
__device__ __forceinline__ uint64_t pk2(float x, float y) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};\n" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ void up2(uint64_t a, float& x, float& y) {
  asm("mov.b64 {%0, %1}, %2;\n" : "=f"(x), "=f"(y) : "l"(a));
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;\n" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;\n" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;\n" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;\n" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// 2F of one cell from its window sums (fa, fb as f32x2 re/im pairs);
// nb2 = (-beta, -beta); k1 = -inf marks a cell that takes no part.
__device__ __forceinline__ float two_f_pairs(uint64_t fa, uint64_t fb, uint64_t nb2, float k1,
                                             float k2, uint64_t tiny2) {
  const uint64_t e = fma2(nb2, fa, fb);
  const uint64_t pa = fma2(fa, fa, tiny2);
  const uint64_t pe = mul2(e, e);
  float a0, a1, e0, e1;
  up2(pa, a0, a1);
  up2(pe, e0, e1);
  return fmaf(k1, a0 + a1, k2 * (e0 + e1));
}

template <bool kShared>
__device__ __forceinline__ void rect_cells_body(const int32_t* __restrict__ i0tab,
    const int32_t* __restrict__ jend, const Coef* __restrict__ coef,
    const float4* __restrict__ px, int32_t n_sft, int32_t n_t0, int32_t n_tau,
    int32_t n_templates, float* __restrict__ map, Partial* __restrict__ parts, int64_t stride,
    uint32_t* __restrict__ err, uint64_t wait_ns, int64_t blk, unsigned char* smem) {
  __shared__ uint64_t s_bar[kSlots];   // one per slot: warp w owns slot w
  __shared__ int4 s_grp[4];   // per group: first row start, row entries, first end, end entries
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tl = rect_tlanes(n_templates);
  const int n_grp = 4 / tl;
  const int st_t = 2 * tl;                      // templates per stage
  const int32_t brows = kGroupRows * n_grp;
  const int32_t n_rb = (n_t0 + brows - 1) / brows;
  const int32_t n_ct = (n_tau + kTileCols - 1) / kTileCols;
  const int32_t n_bc = (n_templates + kBlockTemplates - 1) / kBlockTemplates;
  if (n_bc == 0 || blk >= (int64_t)n_rb * n_ct * n_bc) return;   // whole block
  // Chunks of one block tile are neighbours (coefficients shared through
  // L2); block tiles run down a column (nearby prefix ranges in flight).
  // (The block count fits 31 bits: the launch checks it.)
  const uint32_t ub = (uint32_t)blk;
  const int32_t bc = (int32_t)(ub % (uint32_t)n_bc);
  const uint32_t bt = ub / (uint32_t)n_bc;
  const int32_t ct = (int32_t)(bt / (uint32_t)n_rb), rb = (int32_t)(bt - (uint32_t)ct * (uint32_t)n_rb);
  const int32_t M0 = rb * brows, n0 = ct * kTileCols;
  const int32_t nl = min(n0 + kTileCols, n_tau) - 1;
  const int grp = warp / (2 * tl), wi = warp - grp * 2 * tl;
  const int half = wi / tl, tlane = wi - half * tl;
  const int32_t m0 = M0 + grp * kGroupRows + half * kTileRows;
  const int32_t rows = max(0, min(kTileRows, n_t0 - m0));
  const int64_t wt = (int64_t)ct * ((n_t0 + kTileRows - 1) / kTileRows) + m0 / kTileRows;
  const int64_t cells = (int64_t)n_t0 * n_tau;
  const int64_t np1 = (int64_t)n_sft + 1;
  const int64_t cell0 = (int64_t)m0 * n_tau + n0 + lane;   // lane's cell in row 0, q = 0

  fence_proxy_async_smem();   // earlier generic writes of the stage buffer vs the copies below
  if (tid < n_grp) {
    const int32_t mg = M0 + tid * kGroupRows;
    const int32_t gr = min(kGroupRows, n_t0 - mg);
    int4 e = make_int4(0, 0, 0, 0);
    if (gr > 0) {
      const int32_t ia = i0tab[mg], jmin = jend[(int64_t)mg * n_tau + n0];
      e = make_int4(ia, i0tab[mg + gr - 1] - ia + 1, jmin,
                    jend[(int64_t)(mg + gr - 1) * n_tau + nl] - jmin + 1);
    }
    s_grp[tid] = e;
  }
  if (tid < kSlots) mbar_init(&s_bar[tid], 1);
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  bool staged = true;
  for (int k = 0; k < n_grp; ++k) {
    const int4 e = s_grp[k];
    if (e.y > 0 && (e.y - 1 > kMaxRowSpread || e.y > kRowCap || e.w > kJCap)) staged = false;
  }
  const int4 G = s_grp[grp];

  const uint32_t raw_s = smem_u32(smem);
  const uint32_t q_s0 = raw_s + (uint32_t)kRawBytes;
  const bool col0 = n0 + lane < n_tau, col1 = n0 + lane + 32 < n_tau;
  auto in_grid = [&](int i) { return (i >> 1) < rows && ((i & 1) ? col1 : col0); };
  auto cell_off = [&](int i) { return (int64_t)(i >> 1) * n_tau + 32 * (i & 1); };

  // Byte offsets within a slot's Q of the lane's window ends and row starts.
  uint32_t qo[kLaneCells], ro[kTileRows];
#pragma unroll
  for (int i = 0; i < kLaneCells; ++i) {
    const int32_t j = in_grid(i) ? jend[cell0 + cell_off(i)] : G.z;
    qo[i] = 16u * (uint32_t)(kRowCap + j - G.z);
  }
#pragma unroll
  for (int r = 0; r < kTileRows; ++r)
    ro[r] = rows > 0 ? 16u * (uint32_t)(i0tab[m0 + min(r, rows - 1)] - G.x) : 0u;

  float k1[kLaneCells], k2[kLaneCells];
  uint64_t nb2[kLaneCells];
  int32_t nval = 0;
  auto load_coef = [&](const Coef* __restrict__ cb) {
    int32_t c = 0;
#pragma unroll
    for (int i = 0; i < kLaneCells; ++i) {
      Coef cf{0.0f, 0.0f, 0.0f, 0.0f};
      if (in_grid(i)) cf = cb[cell0 + cell_off(i)];
      const bool ok = cf.valid == 1.0f;
      k1[i] = ok ? cf.k1 : -INFINITY;
      k2[i] = ok ? cf.k2 : 0.0f;
      nb2[i] = pk2(-cf.beta, -cf.beta);
      c += ok ? 1 : 0;
    }
    nval = (int32_t)__reduce_add_sync(0xffffffffu, (unsigned)c);
  };
  if (kShared) load_coef(coef);

  const int32_t t_begin = bc * kBlockTemplates;
  const int32_t t_end = min(n_templates, t_begin + kBlockTemplates);
  const int n_st = (t_end - t_begin + st_t - 1) / st_t;
  // Warp w owns slot w of every stage: the slot's template is the w-th of
  // the stage (wi), its group is the warp's own.  Lane 0 fetches the slot's
  // prefix entries for stage st; the owner rebases them, and the two warps
  // of a (group, template lane) pair, which read each other's slots, meet
  // at a named barrier.
  auto issue = [&](int st) {
    const int32_t tm = t_begin + st * st_t + wi;
    if (lane == 0 && G.y > 0 && tm < t_end) {
      const float4* pt = px + (int64_t)tm * 2 * np1;
      const uint32_t dst = raw_s + (uint32_t)(warp * kSlotEntries * 32);
      mbar_arrive_expect_tx(&s_bar[warp], 32u * (uint32_t)(G.y + G.w));
      bulk_g2s(dst, pt + 2 * (int64_t)G.x, 32u * (uint32_t)G.y, &s_bar[warp]);
      bulk_g2s(dst + kRowCap * 32, pt + 2 * (int64_t)G.z, 32u * (uint32_t)G.w, &s_bar[warp]);
    }
  };
  const int pair_bar = 1 + grp * tl + tlane;   // named barrier of the warp pair (ids 1..4)

  constexpr float kHalfLog2e = 0.72134752044448170368f;   // log2(e) / 2
  const uint64_t tiny2 = pk2(1e-30f, 1e-30f);
  // A warp whose wait gave up (its own limit, or another block's timeout)
  // first lets the copy of that stage land (bounded by kWaitNs), then issues
  // no more copies and skips its work; it still meets its pair's named
  // barrier every stage.  The call's outputs are then undefined and the
  // plan's status reports the timeout.
  bool dead = false;
  if (staged) issue(0);
  for (int st = 0; st < n_st; ++st) {
    const uint32_t qs = q_s0 + (uint32_t)((st & 1) * kQBytes);
    if (staged) {
      if (!dead && G.y > 0 && t_begin + st * st_t + wi < t_end) {
        const bool got = mbar_wait_or_abort(&s_bar[warp], (uint32_t)(st & 1), err, wait_ns);
        if (!__all_sync(0xffffffffu, got)) {
          mbar_wait_bounded(&s_bar[warp], (uint32_t)(st & 1), kWaitNs);
          __syncwarp();
          dead = true;
        }
      }
      if (!dead && G.y > 0 && t_begin + st * st_t + wi < t_end) {
        const uint32_t rs = raw_s + (uint32_t)(warp * kSlotEntries * 32);
        const uint32_t qd = qs + (uint32_t)(warp * kSlotEntries * 16);
        uint64_t hb0, hb1, lb0, lb1;
        lds_pairs(rs, hb0, hb1);
        lds_pairs(rs + 16, lb0, lb1);
        auto rebase = [&](int e) {
          uint64_t h0, h1, l0, l1;
          lds_pairs(rs + 32 * e, h0, h1);
          lds_pairs(rs + 32 * e + 16, l0, l1);
          const uint64_t q0 = add2(sub2(h0, hb0), sub2(l0, lb0));
          const uint64_t q1 = add2(sub2(h1, hb1), sub2(l1, lb1));
          asm volatile("st.shared.v2.b64 [%0], {%1, %2};\n" ::"r"(qd + (uint32_t)(e * 16)),
                       "l"(q0), "l"(q1) : "memory");
        };
        for (int e = lane; e < G.y; e += 32) rebase(e);
        for (int e = kRowCap + lane; e < kRowCap + G.w; e += 32) rebase(e);
        fence_proxy_async_smem();   // the reads of raw above vs the next copy into it
        __syncwarp();
        if (st + 1 < n_st) issue(st + 1);
      }
      asm volatile("bar.sync %0, 64;" ::"r"(pair_bar) : "memory");
    }
    if (rows == 0 || dead) continue;   // warp below the grid, or given up: barriers only
    for (int g = tlane; g < st_t; g += tl) {
      const int32_t tm = t_begin + st * st_t + g;
      if (tm >= t_end) break;
      if (!kShared) load_coef(coef + (int64_t)tm * cells);
      float v[kLaneCells];
      if (staged) {
        const uint32_t sq = qs + (uint32_t)((grp * st_t + g) * kSlotEntries * 16);
#pragma unroll
        for (int r = 0; r < kTileRows; ++r) {
          uint64_t ia, ib;
          lds_pairs(sq + ro[r], ia, ib);
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int i = 2 * r + q;
            uint64_t ja, jb;
            lds_pairs(sq + qo[i], ja, jb);
            v[i] = two_f_pairs(sub2(ja, ia), sub2(jb, ib), nb2[i], k1[i], k2[i], tiny2);
          }
        }
      } else {
        // Window sums from the float pairs in global memory, parked in the
        // warp's part of the (unused) stage buffer.
        const float4* pt = px + (int64_t)tm * 2 * np1;
        const uint32_t wb = raw_s + (uint32_t)(warp * kLaneCells * 32 * 16 + lane * 16);
        __syncwarp();
#pragma unroll 1
        for (int i = 0; i < kLaneCells; ++i) {
          const int32_t i0 = i0tab[m0 + min(i >> 1, rows - 1)];
          const int32_t j = in_grid(i) ? jend[cell0 + cell_off(i)] : i0;
          const float4 hi = pt[2 * (int64_t)i0], li = pt[2 * (int64_t)i0 + 1];
          const float4 hj = pt[2 * (int64_t)j], lj = pt[2 * (int64_t)j + 1];
          const uint64_t a = add2(sub2(pk2(hj.x, hj.y), pk2(hi.x, hi.y)), sub2(pk2(lj.x, lj.y), pk2(li.x, li.y)));
          const uint64_t b = add2(sub2(pk2(hj.z, hj.w), pk2(hi.z, hi.w)), sub2(pk2(lj.z, lj.w), pk2(li.z, li.w)));
          asm volatile("st.shared.v2.b64 [%0], {%1, %2};\n" ::"r"(wb + (uint32_t)(i * 32 * 16)),
                       "l"(a), "l"(b) : "memory");
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < kLaneCells; ++i) {
          uint64_t a, b;
          lds_pairs(wb + (uint32_t)(i * 32 * 16), a, b);
          v[i] = two_f_pairs(a, b, nb2[i], k1[i], k2[i], tiny2);
        }
      }
      const float mx = fmaxf(fmaxf(fmaxf(v[0], v[1]), fmaxf(v[2], v[3])),
                             fmaxf(fmaxf(v[4], v[5]), fmaxf(v[6], v[7])));
      if (map) {
        float* mr = map + (int64_t)tm * cells + cell0;
        if (rows == kTileRows && col1) {
#pragma unroll
          for (int r = 0; r < kTileRows; ++r, mr += n_tau) {
            st_stream(mr, fmaxf(v[2 * r], 0.0f));
            st_stream(mr + 32, fmaxf(v[2 * r + 1], 0.0f));
          }
        } else {
#pragma unroll
          for (int i = 0; i < kLaneCells; ++i)
            if (in_grid(i)) st_stream(mr + cell_off(i), fmaxf(v[i], 0.0f));
        }
      }
      // 2F >= 0, so its bit pattern orders like the value; 0 marks "no valid cell".
      const unsigned mu = __reduce_max_sync(0xffffffffu, mx >= 0.0f ? __float_as_uint(mx) + 1u : 0u);
      if (mu == 0u) {
        if (lane == 0) parts[(int64_t)tm * stride + wt] = partial_empty();
        continue;
      }
      const float M = __uint_as_float(mu - 1u);
      const float mc = -M * kHalfLog2e;
      float e[kLaneCells];
#pragma unroll
      for (int i = 0; i < kLaneCells; ++i) e[i] = ex2_approx(fmaf(v[i], kHalfLog2e, mc));
      // The lane's sum is in [0, 8] (every term <= 1); summed over the warp in
      // 2^-23 fixed point by an integer reduction (absolute error <= 32 x
      // 2^-24 against a sum >= 1, the maximum cell's own term).
      const float sl = ((e[0] + e[1]) + (e[2] + e[3])) + ((e[4] + e[5]) + (e[6] + e[7]));
      const unsigned sfix = __reduce_add_sync(0xffffffffu, __float2uint_rn(sl * 8388608.0f));
      // Only lanes holding the maximum look for their first cell at it.
      unsigned cand = (unsigned)kNoArg;
      if (mx == M) {
#pragma unroll
        for (int i = kLaneCells - 1; i >= 0; --i)
          if (v[i] == M) cand = (unsigned)(cell0 + cell_off(i));
      }
      const int32_t arg = (int32_t)__reduce_min_sync(0xffffffffu, cand);
      if (lane == 0) {
        const float4 pv = make_float4(M, __int_as_float(arg), (float)sfix * (1.0f / 8388608.0f),
                                      __int_as_float(nval));
        *reinterpret_cast<float4*>(parts + (int64_t)tm * stride + wt) = pv;
      }
    }
  }
  __syncthreads();   // every wait on the mbarriers is done before they are retired
  if (tid < kSlots) mbar_inval(&s_bar[tid]);
}

template <bool kShared>
__global__ void __launch_bounds__(kCellThreads, 2)
k_rect_cells(const int32_t* __restrict__ i0tab, const int32_t* __restrict__ jend,
             const Coef* __restrict__ coef, const float4* __restrict__ px, int32_t n_sft,
             int32_t n_t0, int32_t n_tau, int32_t n_templates, float* __restrict__ map,
             Partial* __restrict__ parts, int64_t stride, uint32_t* __restrict__ err,
             uint64_t wait_ns) {
  extern __shared__ __align__(128) unsigned char s_cells[];
  rect_cells_body<kShared>(i0tab, jend, coef, px, n_sft, n_t0, n_tau, n_templates, map, parts,
                           stride, err, wait_ns, blockIdx.x, s_cells);
}

int64_t rect_partial_slots(const fmap_grid& g, int32_t, int32_t) { return rect_tiles(g); }
int64_t rect_cells_blocks(const fmap_grid& g, int32_t n_templates, int32_t) {
  return rect_cmaj_blocks(g, n_templates);
}
size_t rect_cells_smem(int32_t, int32_t) { return rect_cmaj_smem(); }

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
    k_rect_scan_antenna<<<n_ant, kScanThreads, 0, s>>>(a->antenna, p->n_sft, (P4*)p->ws.pa);
  } else {
    cudaMemsetAsync(p->ws.pa, 0, sizeof(P4) * n_ant, s);
  }
  const int64_t total = cells * n_ant;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)p->n_sm * 16);
  k_rect_coef<<<blocks, 256, 0, s>>>(p->ws.i0, p->ws.jend, (const P4*)p->ws.pa, p->n_sft, g.n_t0,
                                     g.n_tau, n_ant, p->ws.coef, p->ws.flag_bits);
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
    p->tiles = TileGeom{0, kRowThreads, g.n_tau, (int32_t)grid.x, 1};
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
  const int32_t T = p->n_templates, sh = a->shared_antenna ? 1 : 0;
  *tiles_used = rect_partial_slots(g, T, sh);
  p->tiles = TileGeom{1, kTileRows, kTileCols, (g.n_t0 + kTileRows - 1) / kTileRows,
                      (g.n_tau + kTileCols - 1) / kTileCols};
  const int64_t blocks = rect_cells_blocks(g, T, sh);
  if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  const size_t smem = rect_cells_smem(T, sh);
  const void* kfn = sh ? (const void*)k_rect_cells<true> : (const void*)k_rect_cells<false>;
  e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (sh)
    k_rect_cells<true><<<(unsigned)blocks, kCellThreads, smem, s>>>(
        p->ws.i0, p->ws.jend, p->ws.coef, p->ws.px, p->n_sft, g.n_t0, g.n_tau, T,
        d_2F, p->ws.partials, p->part_stride, p->ws.dev_err, (uint64_t)p->wait_ns);
  else
    k_rect_cells<false><<<(unsigned)blocks, kCellThreads, smem, s>>>(
        p->ws.i0, p->ws.jend, p->ws.coef, p->ws.px, p->n_sft, g.n_t0, g.n_tau, T,
        d_2F, p->ws.partials, p->part_stride, p->ws.dev_err, (uint64_t)p->wait_ns);
  p->launches += 1;
  return cudaGetLastError();
}


// ---- persistent multi-instance dispatchers (uneven batches) ----
__global__ void __launch_bounds__(kScanThreads) kb_rect_ant(const BItem* __restrict__ items,
                                                            BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    rect_scan_antenna_body(it.antenna, it.n_sft, (P4*)it.pa, make_uint3((unsigned)k, 0, 0),
                           dim3((unsigned)it.n_ant));
  });
}
__global__ void __launch_bounds__(256) kb_rect_coef(const BItem* __restrict__ items, BUnits u) {
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    const unsigned nb = (unsigned)((it.cells * it.n_ant + 255) / 256);
    for (int q = 0; q < kCoefBlocksPerUnit; ++q)
      rect_coef_body(it.i0, it.jend, (const P4*)it.pa, it.n_sft, it.g.n_t0, it.g.n_tau, it.n_ant,
                     it.coef, it.flag_bits, make_uint3((unsigned)(k * kCoefBlocksPerUnit + q), 0, 0),
                     dim3(nb));
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
  extern __shared__ __align__(128) unsigned char s_cells[];
  batch_loop(items, u, [&](const BItem& it, int64_t k) {
    if (it.shared)
      rect_cells_body<true>(it.i0, it.jend, it.coef, it.px, it.n_sft, it.g.n_t0, it.g.n_tau,
                            it.T, it.map, it.partials, it.part_stride, it.dev_err, kWaitNs, k,
                            s_cells);
    else
      rect_cells_body<false>(it.i0, it.jend, it.coef, it.px, it.n_sft, it.g.n_t0, it.g.n_tau,
                             it.T, it.map, it.partials, it.part_stride, it.dev_err, kWaitNs, k,
                             s_cells);
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
