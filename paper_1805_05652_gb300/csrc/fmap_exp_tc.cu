// Exponential-window contraction on the 5th-generation tensor cores (tcgen05).
//
// S[(m, n), c] = sum_a W[(m, n), a] X[a, c] with W = e^{-(t_a - t0_m)/tau_n}
// inside the window (Eq. winexp) and X = the 4T data columns (Re Fa, Im Fa,
// Re Fb, Im Fb of each template).  A tile is 128 cells (one t0 row, 128
// consecutive tau) x N data columns (N = 4 x templates of the chunk, <= 256).
//
// Per K-tile of KT atoms (128 bytes of one operand row):
//   * eight "generator" warps compute W for their rows in registers (one
//     exp2 per element), split it into hi + lo (TF32 or BF16) and store both
//     into tensor memory, which is the MMA's A operand;
//   * one warp streams the hi and lo K-major X tiles into shared memory with
//     TMA (128-byte swizzle), the MMA's B operand;
//   * one thread issues hi*hi + hi*lo + lo*hi (3 MMAs per K step) into an
//     FP32 accumulator in tensor memory; tcgen05.commit frees the stage.
// Then the generator warps read the accumulator back (tcgen05.ld), apply the
// per-cell FP64-derived 2F coefficients, write the map and the per-template
// (max, argmax, log-sum-exp) partials.  K-tiles outside the union of the
// tile's windows are never visited; W is zero outside each cell's window.
//
// Every wait on an mbarrier is bounded by %globaltimer; on expiry the kernel
// latches an error bit in the plan's status word and winds down.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include "fmap_device.cuh"

namespace fmap {
namespace tc {

constexpr int kGenWarps = 8;
constexpr int kMmaWarp = 8;
constexpr int kTmaWarp = 9;
constexpr int kThreads = 320;
constexpr int kRows = 128;
constexpr int kAColsPerStage = 64;   // hi (32 columns) + lo (32 columns)
constexpr int kDtCap = 4096;          // atoms of relative times staged per refill (16 KB)
constexpr float kFar = 1.0e30f;       // relative time of atoms outside every window

// ---------------------------------------------------------------- PTX ------
// Bounded wait; false on timeout (limit_ns; 0: at the first incomplete
// poll) or when another role already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                          uint64_t limit_ns) {
  if (limit_ns == 0) return mbar_test_wait(bar, parity);
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (*abort) return false;
    if (globaltimer() - t0 > limit_ns) return false;
    if (mbar_try_wait(bar, parity)) return true;
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// The three products of one MMA K step, hi*hi (accumulating if acc != 0),
// hi*lo and lo*hi, into the accumulator at d; the B descriptors are given as
// their low words (start address) and the common high word.
template <bool BF16>
__device__ __forceinline__ void mma_kstep(uint32_t d, uint32_t a_hi, uint32_t a_lo,
                                          uint32_t bh_lo, uint32_t bl_lo, uint32_t b_hi32,
                                          uint32_t idesc, uint32_t acc) {
  if constexpr (BF16) {
    asm volatile(
        "{\n .reg .pred p, t;\n .reg .b64 bh, bl;\n setp.ne.b32 p, %7, 0;\n"
        " setp.eq.b32 t, %6, %6;\n mov.b64 bh, {%3, %5};\n mov.b64 bl, {%4, %5};\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], bh, %6, p;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], bl, %6, t;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%2], bh, %6, t;\n}" ::"r"(d),
        "r"(a_hi), "r"(a_lo), "r"(bh_lo), "r"(bl_lo), "r"(b_hi32), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p, t;\n .reg .b64 bh, bl;\n setp.ne.b32 p, %7, 0;\n"
        " setp.eq.b32 t, %6, %6;\n mov.b64 bh, {%3, %5};\n mov.b64 bl, {%4, %5};\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], bh, %6, p;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], bl, %6, t;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%2], bh, %6, t;\n}" ::"r"(d),
        "r"(a_hi), "r"(a_lo), "r"(bh_lo), "r"(bl_lo), "r"(b_hi32), "r"(idesc), "r"(acc)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
  return y;
}
// Pack (lo_elem -> bits 15:0, hi_elem -> bits 31:16) as bf16x2, round to nearest.
__device__ __forceinline__ uint32_t pack_bf16(float even, float odd) {
  uint32_t y;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(y) : "f"(odd), "f"(even));
  return y;
}
__device__ __forceinline__ void mul_x2(float& r0, float& r1, float a0, float a1, float b) {
  asm("{\n.reg .b64 a, b, d;\nmov.b64 a, {%2, %3};\nmov.b64 b, {%4, %4};\n"
      "mul.rn.f32x2 d, a, b;\nmov.b64 {%0, %1}, d;\n}"
      : "=f"(r0), "=f"(r1)
      : "f"(a0), "f"(a1), "f"(b));
}
__device__ __forceinline__ void sub_x2(float& r0, float& r1, float a0, float a1, float b0,
                                       float b1) {
  asm("{\n.reg .b64 a, b, d;\nmov.b64 a, {%2, %3};\nmov.b64 b, {%4, %5};\n"
      "sub.rn.f32x2 d, a, b;\nmov.b64 {%0, %1}, d;\n}"
      : "=f"(r0), "=f"(r1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes in 8-row (1024-byte) groups.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;            // leading-dimension offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride between 8-row groups
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulate, A/B both TF32 or both BF16,
// K-major A and B, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_of(bool bf16, int n) {
  return (1u << 4) | ((bf16 ? 1u : 2u) << 7) | ((bf16 ? 1u : 2u) << 10) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

struct Params {
  const int32_t* rel_t;
  const int64_t* t_base;
  fmap_grid g;
  const int64_t* ax;   // grid values: t0_m, then tau_n
  const float2* wtab;  // FMAP_TABLE grids: the window table (n_tab samples + sentinel)
  int32_t n_tab;
  const int32_t* i0tab;
  const int32_t* jend;
  const Coef* coef;
  int32_t shared_antenna;
  int32_t n_templates;
  int32_t n_cols;      // N of this launch (multiple of 64, <= 256)
  int32_t tmem_cols;   // power of two >= 2 n_cols + NS * kAColsPerStage
  int32_t nblk;        // 128-cell blocks per t0 row
  float* map;
  Partial* parts;
  int64_t stride;
  uint32_t* err;
  uint64_t wait_ns;    // limit of the pipeline's waits (the drains take kWaitNs)
};

// Accumulation in chunks.  A tensor-core MMA adds its products to the FP32
// accumulator with truncation (no round to nearest), which biases a long sum
// towards zero by a few ulp per MMA: over the ~10^2-10^3 MMAs of a long window
// the sums shrink by ~1e-5 relative, and so does every 2F (measured: the log
// Bayes factor of pure-noise maps of 5000 SFTs off by 1-3e-4 with 256-atom
// chunks).  So every K-tile (32 or 64 atoms, 12 MMAs) is a chunk of its own,
// alternately in two TMEM accumulators; the generator warps add a finished
// chunk's accumulator, with round-to-nearest FP32 additions, to running sums
// in shared memory just before they fill the first stage of the chunk two
// later, which is when the MMA thread needs that accumulator again.
constexpr int kChunkTiles = 1;

// TAB: weights from the window table (FMAP_TABLE grids) instead of exp2; the
// table sits in shared memory after the staged relative times.
// (at most 102 registers a thread, so that two CTAs fit an SM's register
// file where their TMEM and shared memory let them.)  RS: the running sums in
// registers (N = 64: 32 a thread), else in shared memory.
template <bool BF16, bool TAB, int NS, bool RS>
__global__ void __launch_bounds__(kThreads, 2)
k_exp_tc(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
         const Params p) {
  constexpr int KT = BF16 ? 64 : 32;          // atoms per K-tile (128-byte operand rows)
  constexpr int HALF = KT / 2;                // atoms per generator warp and K-tile
  constexpr int KSTEP = BF16 ? 16 : 8;        // atoms per MMA
  constexpr int NKS = KT / KSTEP;             // MMAs per product and K-tile
  constexpr int P = kChunkTiles;              // K-tiles per accumulation chunk
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int kStages = NS;                 // A/B pipeline stages
  float* s_dt = (float*)(smem + (size_t)kStages * 2 * p.n_cols * 128);
  float2* s_tab = (float2*)(s_dt + kDtCap);   // TAB only
  // running sums [N / 4][128 rows] float4 (column quads of each row)
  float4* s_sum = (float4*)(((uintptr_t)(s_tab + (TAB ? kTabMax + 1 : 0)) + 15) & ~(uintptr_t)15);
  __shared__ uint64_t bar_full_b[kStages], bar_full_a[kStages], bar_empty[kStages];
  __shared__ uint64_t bar_accf[2], bar_drain[2], bar_final;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ int32_t s_jmax;
  __shared__ Partial s_red[4][64];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = p.n_cols;
  const uint32_t op_bytes = (uint32_t)N * 128u;
  const fmap_grid& g = p.g;
  const int32_t nb = p.nblk - 1 - (int32_t)(blockIdx.x / g.n_t0);   // heavy tiles first
  const int32_t m = (int32_t)(blockIdx.x % g.n_t0);
  const int chunk = blockIdx.y;
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const int64_t tile = (int64_t)m * p.nblk + nb;
  const int32_t i0 = p.i0tab[m];

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&bar_full_b[s], 1);
      mbar_init(&bar_full_a[s], kGenWarps);
      mbar_init(&bar_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_accf[b], 1);
      mbar_init(&bar_drain[b], kGenWarps);
    }
    mbar_init(&bar_final, 1);
    s_abort = 0;
    s_jmax = i0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp < 4) {
    const int32_t n = nb * kRows + warp * 32 + lane;
    const int32_t jc = n < g.n_tau ? p.jend[(int64_t)m * g.n_tau + n] : i0;
    const int32_t jw = __reduce_max_sync(0xffffffffu, jc);
    if (lane == 0) atomicMax(&s_jmax, jw);
  }
  if (warp == 0) tmem_alloc(&s_tmem, (uint32_t)p.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int32_t jmax = s_jmax;
  const int32_t k_begin = (i0 / KT) * KT;
  const int n_kt = jmax > i0 ? (jmax - k_begin + KT - 1) / KT : 0;
  const int n_chunks = (n_kt + P - 1) / P;
  const uint32_t a_col0 = 2u * (uint32_t)N;   // A stages follow the two accumulators

  if (warp == kTmaWarp) {
    // ---------------- TMA producer of the X tiles ----------------
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < n_kt; ++it) {
        const int s = it % kStages;
        if (it >= kStages &&
            !mbar_wait(&bar_empty[s], ((it / kStages) + 1) & 1, &s_abort, p.wait_ns)) {
          atomicExch(&s_abort, 1);
          break;
        }
        if (s_abort) break;
        uint8_t* dst = smem + (size_t)s * 2 * op_bytes;
        mbar_arrive_expect_tx(&bar_full_b[s], 2 * op_bytes);
        tma_load_2d(dst, &tm_hi, &bar_full_b[s], k_begin + it * KT, chunk * N);
        tma_load_2d(dst + op_bytes, &tm_lo, &bar_full_b[s], k_begin + it * KT, chunk * N);
        issued = it + 1;
      }
      if (s_abort) {
        // let the copies already in flight land before the block exits
        for (int it = issued - kStages > 0 ? issued - kStages : 0; it < issued; ++it) {
          volatile int never = 0;
          mbar_wait(&bar_full_b[it % kStages], (it / kStages) & 1, &never, kWaitNs);
        }
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    // One thread issues every MMA of the CTA, so work added to its loop delays
    // them all: stage, phase, chunk, TMEM column and descriptor address
    // advance by additions, and no descriptor is rebuilt per K-tile.  (The
    // descriptor's start-address field, bits 0-13 = address / 16, cannot
    // carry into the next field: shared memory ends below 2^18 bytes.)
    if (lane == 0) {
      const uint32_t idesc = idesc_of(BF16, N);
      const uint64_t d0 = sdesc_sw128(smem_u32(smem));
      const uint32_t d_lo0 = (uint32_t)d0, d_hi = (uint32_t)(d0 >> 32);
      const uint32_t op16 = op_bytes >> 4, stage16 = (2 * op_bytes) >> 4;
      uint32_t d_lo = d_lo0, a_st = tmem + a_col0, par = 0;
      int s = 0, kc = 0, c = 0;                 // stage, K-tile within the chunk, chunk
      uint32_t acc = tmem;                      // accumulator of chunk c (column (c & 1) N)
      bool issued = false;
      for (int it = 0; it < n_kt; ++it) {
        // a chunk reuses the accumulator of chunk c - 2 once it is drained
        if (kc == 0 && c >= 2 &&
            !mbar_wait(&bar_drain[c & 1], ((c - 2) >> 1) & 1, &s_abort, p.wait_ns)) {
          atomicExch(&s_abort, 1);
          break;
        }
        if (!mbar_wait(&bar_full_b[s], par, &s_abort, p.wait_ns) ||
            !mbar_wait(&bar_full_a[s], par, &s_abort, p.wait_ns)) {
          atomicExch(&s_abort, 1);
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int ks = 0; ks < NKS; ++ks) {
          // 8 TMEM columns and 32 bytes of the B rows per MMA K step
          const uint32_t ac = (uint32_t)(ks * 8), bk = (uint32_t)((ks * 32) >> 4);
          mma_kstep<BF16>(acc, a_st + ac, a_st + 32u + ac, d_lo + bk, d_lo + op16 + bk, d_hi,
                          idesc, (kc > 0 || ks > 0) ? 1u : 0u);
        }
        issued = true;
        mma_commit(&bar_empty[s]);
        if (++kc == P || it + 1 == n_kt) {
          mma_commit(&bar_accf[c & 1]);
          kc = 0;
          ++c;
          acc = tmem + (uint32_t)((c & 1) * N);
        }
        if (++s == kStages) {
          s = 0;
          par ^= 1u;
          d_lo = d_lo0;
          a_st = tmem + a_col0;
        } else {
          d_lo += stage16;
          a_st += (uint32_t)kAColsPerStage;
        }
      }
      if (issued) {
        // every MMA this thread issued completes before the block releases its
        // tensor memory, also after a wait gave up
        mma_commit(&bar_final);
        volatile int never = 0;
        mbar_wait(&bar_final, 0, &never, kWaitNs);
      }
    }
  } else {
    // ---------------- W generators, then the epilogue ----------------
    const int q = warp & 3, h = warp >> 2;
    const int row = q * 32 + lane;
    const int32_t n = nb * kRows + row;
    const bool in_grid = n < g.n_tau;
    const int64_t cell = (int64_t)m * g.n_tau + (in_grid ? n : 0);
    const int32_t jc = in_grid ? p.jend[cell] : i0;
    // -log2(e) / tau by an FP32 division (within 1.5 ulp; FP64 runs at 1/64
    // of the FP32 rate on GB300)
    const float c2 = -1.44269504088896341f / (float)grid_tau(g, p.ax, (in_grid ? n : 0));
    int32_t t0rel = 0;
    if (jmax > i0) t0rel = (int32_t)(grid_t0(g, p.ax, m) - *p.t_base);
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int gtid = threadIdx.x;          // 0 .. 255 over the generator warps
    const int ncol = N / 2;                // this warp's accumulator columns
    const uint32_t col_h = (uint32_t)(h * ncol);
    float su = 0.0f;                       // TAB: table samples per second of t - t0
    if constexpr (TAB) {
      su = (float)tab_scale(p.n_tab, exp_cut8_of(g), grid_tau(g, p.ax, (in_grid ? n : 0)));
      for (int k = gtid; k <= p.n_tab; k += kGenWarps * 32) s_tab[k] = p.wtab[k];
      asm volatile("bar.sync 1, %0;" ::"n"(kGenWarps * 32) : "memory");
    }
    bool ok_run = true;
    int drained = 0;                       // chunks added to the running sums
    float rs[RS ? 32 : 1];                 // RS: this thread's 32 running sums
#pragma unroll
    for (int i = 0; i < (RS ? 32 : 1); ++i) rs[i] = 0.0f;
    // Adds chunk c's accumulator (this thread's row, this warp's columns) to
    // the running sums (the first chunk initialises them), then releases the
    // accumulator to the MMA thread.
    auto drain = [&](int c) -> bool {
      if (!mbar_wait(&bar_accf[c & 1], (c >> 1) & 1, &s_abort, p.wait_ns)) return false;
      tc_fence_after();
      const uint32_t base = tmem + lane_off + (uint32_t)((c & 1) * N) + col_h;
      if constexpr (RS) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          float v[16];
          tmem_ld16(base + (uint32_t)(16 * q), v);
#pragma unroll
          for (int i = 0; i < 16; ++i) rs[16 * q + i] += v[i];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_drain[c & 1]);
        return true;
      }
#pragma unroll 1
      for (int g8 = 0; g8 < ncol; g8 += 16) {
        float v[16];
        tmem_ld16(base + (uint32_t)g8, v);
        float4* sp = s_sum + (size_t)((col_h + g8) >> 2) * kRows + row;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float4 o = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
          if (c > 0) {
            const float4 r = sp[(size_t)i * kRows];
            o.x += r.x;
            o.y += r.y;
            o.z += r.z;
            o.w += r.w;
          }
          sp[(size_t)i * kRows] = o;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_drain[c & 1]);
      return true;
    };
    for (int it = 0; it < n_kt; ++it) {
      const int s = it % kStages;
      const int pos = (it * KT) % kDtCap;
      if (pos == 0) {
        // Stage the next kDtCap atoms' times relative to t0 (shared by all 128
        // rows of the tile).  Atoms before the tile's t0 or past the union of
        // its windows get kFar, whose weight ex2(c2 kFar) underflows to 0.
        asm volatile("bar.sync 1, %0;" ::"n"(kGenWarps * 32) : "memory");
        for (int idx = gtid; idx < kDtCap; idx += kGenWarps * 32) {
          const int32_t a = k_begin + it * KT + idx;
          float v = kFar;
          if (a >= i0 && a < jmax) v = (float)(p.rel_t[a] - t0rel);
          s_dt[idx] = v;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kGenWarps * 32) : "memory");
      }
      // after a timeout keep looping (without work) so that every generator
      // warp reaches the same shared-memory barriers
      if (!ok_run || s_abort) continue;
      if (it >= kStages &&
          !mbar_wait(&bar_empty[s], ((it / kStages) + 1) & 1, &s_abort, p.wait_ns)) {
        atomicExch(&s_abort, 1);
        ok_run = false;
        continue;
      }
      // before the first stage of chunk c, add chunk c - 2 to the running
      // sums: the MMA thread reuses its accumulator for chunk c (its MMAs
      // only needed stages already filled, so the wait for them ends)
      if (it % P == 0 && it / P >= 2) {
        if (!drain(drained)) {
          atomicExch(&s_abort, 1);
          ok_run = false;
          continue;
        }
        ++drained;
      }
      const int32_t a0 = k_begin + it * KT + h * HALF;
      const int32_t cnt = jc - a0;                     // leading atoms inside this row's window
      const uint32_t col = a_col0 + (uint32_t)(s * kAColsPerStage + h * 16);
      // two passes of Q atoms (fewer live registers): W, its hi + lo split,
      // and QW words of each operand into the stage's columns
      constexpr int Q = HALF / 2;
      constexpr int QW = BF16 ? Q / 2 : Q;
      static_assert(QW == 8, "eight 32-bit words per operand and pass");
      const bool none = __all_sync(0xffffffffu, cnt <= 0);
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        uint32_t vhi[QW], vlo[QW];
        if (none) {
#pragma unroll
          for (int j = 0; j < QW; ++j) vhi[j] = vlo[j] = 0u;
        } else {
          float w[Q];
          const float4* dp = reinterpret_cast<const float4*>(s_dt + pos + h * HALF + part * Q);
#pragma unroll
          for (int v = 0; v < Q / 4; ++v) {
            const float4 d4 = dp[v];
            if constexpr (TAB) {
              w[4 * v] = tab_weight(su * d4.x, s_tab, p.n_tab);
              w[4 * v + 1] = tab_weight(su * d4.y, s_tab, p.n_tab);
              w[4 * v + 2] = tab_weight(su * d4.z, s_tab, p.n_tab);
              w[4 * v + 3] = tab_weight(su * d4.w, s_tab, p.n_tab);
            } else {
              float e0, e1, e2, e3;
              mul_x2(e0, e1, d4.x, d4.y, c2);
              mul_x2(e2, e3, d4.z, d4.w, c2);
              w[4 * v] = ex2(e0);
              w[4 * v + 1] = ex2(e1);
              w[4 * v + 2] = ex2(e2);
              w[4 * v + 3] = ex2(e3);
            }
          }
          const int32_t cq = cnt - part * Q;
          if (!__all_sync(0xffffffffu, cq >= Q)) {
#pragma unroll
            for (int j = 0; j < Q; ++j) w[j] = j < cq ? w[j] : 0.0f;
          }
          if constexpr (BF16) {
#pragma unroll
            for (int j = 0; j < QW; ++j) {
              const uint32_t hp = pack_bf16(w[2 * j], w[2 * j + 1]);
              const float he = __uint_as_float(hp << 16), ho = __uint_as_float(hp & 0xffff0000u);
              float le, lo;
              sub_x2(le, lo, w[2 * j], w[2 * j + 1], he, ho);
              vhi[j] = hp;
              vlo[j] = pack_bf16(le, lo);
            }
          } else {
            // the MMA reads TF32 operands as FP32 bit patterns and ignores the
            // low 13 bits, so the remainder needs no conversion of its own
#pragma unroll
            for (int j = 0; j < QW; ++j) {
              const uint32_t hb = to_tf32(w[j]);
              vhi[j] = hb;
              vlo[j] = __float_as_uint(w[j] - __uint_as_float(hb));
            }
          }
        }
        tmem_st8(tmem + lane_off + col + (uint32_t)(part * QW), vhi);
        tmem_st8(tmem + lane_off + col + 32u + (uint32_t)(part * QW), vlo);
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_full_a[s]);
    }
    // ---- epilogue: running sums + the chunks still in TMEM -> 2F ----
    // (the last two chunks are still undrained; their MMAs finish before the
    // accumulators are read)
    bool have_acc = n_kt > 0 && ok_run;
    for (int c = drained; have_acc && c < n_chunks; ++c)
      if (!mbar_wait(&bar_accf[c & 1], (c >> 1) & 1, &s_abort, p.wait_ns)) {
        atomicExch(&s_abort, 1);
        have_acc = false;
      }
    tc_fence_after();
    const int tmpl_per_warp = N / 8;          // this half's templates
    const Coef cf0 = p.coef[cell];
    for (int g8 = 0; g8 < tmpl_per_warp; g8 += 8) {
      float acc[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] = 0.0f;
      if (have_acc) {
        if (RS && drained > 0) {
#pragma unroll
          for (int i = 0; i < (RS ? 32 : 1); ++i) acc[i] = rs[i];
        } else if (drained > 0) {
          const float4* sp = s_sum + (size_t)((col_h + g8 * 4) >> 2) * kRows + row;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float4 r = sp[(size_t)i * kRows];
            acc[4 * i] = r.x;
            acc[4 * i + 1] = r.y;
            acc[4 * i + 2] = r.z;
            acc[4 * i + 3] = r.w;
          }
        }
#pragma unroll 1
        for (int c = drained; c < n_chunks; ++c) {
          const uint32_t ca = tmem + lane_off + (uint32_t)((c & 1) * N) + col_h + (uint32_t)(g8 * 4);
          float v[16];
          tmem_ld16(ca, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[i] += v[i];
          tmem_ld16(ca + 16u, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[16 + i] += v[i];
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int tl = h * tmpl_per_warp + g8 + k;       // template within the chunk
        const int32_t tq = chunk * (N / 4) + tl;
        if (g8 + k >= tmpl_per_warp) break;
        const bool exists = tq < p.n_templates;
        const Coef cf = (p.shared_antenna || !exists) ? cf0 : p.coef[(int64_t)tq * cells + cell];
        const float v = two_f(cf, acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
        const bool ok = in_grid && exists && cf.valid == 1.0f;
        if (p.map && in_grid && exists && cf.valid != 2.0f)
          p.map[(int64_t)tq * cells + cell] = ok ? v : 0.0f;
        // The warp's partial over its 32 cells by integer reductions: the
        // maximum over the 2F bit patterns (2F >= 0; 0 = no valid cell), the
        // exp-terms in 2^-26 fixed point (each <= 1, the sum >= 1), the
        // lowest cell index at the maximum, the valid count.
        const unsigned mu = __reduce_max_sync(0xffffffffu, ok ? __float_as_uint(v) + 1u : 0u);
        Partial pt = partial_empty();
        if (mu != 0u) {
          const float M = __uint_as_float(mu - 1u);
          const float e = ok ? __expf(0.5f * (v - M)) : 0.0f;
          const unsigned sfix = __reduce_add_sync(0xffffffffu, __float2uint_rn(e * 67108864.0f));
          pt.max2F = M;
          pt.arg = (int32_t)__reduce_min_sync(0xffffffffu,
                                              ok && v == M ? (unsigned)cell : (unsigned)kNoArg);
          pt.sum = (float)sfix * (1.0f / 67108864.0f);
          pt.nvalid = (int32_t)__reduce_add_sync(0xffffffffu, ok ? 1u : 0u);
        }
        if (lane == 0) s_red[q][tl] = pt;
      }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kGenWarps * 32) : "memory");
    const int gt = threadIdx.x;              // 0 .. 255
    if (gt < N / 4) {
      const int32_t tq = chunk * (N / 4) + gt;
      if (tq < p.n_templates) {
        Partial r = partial_merge(partial_merge(s_red[0][gt], s_red[1][gt]),
                                  partial_merge(s_red[2][gt], s_red[3][gt]));
        p.parts[(int64_t)tq * p.stride + tile] = r;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (s_abort && threadIdx.x == 0) atomicOr(p.err, DEV_ERR_TIMEOUT);
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)p.tmem_cols);
  }
}

// Split X into hi + lo operands ([4T][n_pad], zero padded): TF32 (stored as
// FP32 bit patterns with 13 low zero bits) or BF16.
template <bool BF16>
__global__ void k_split_x(const float* __restrict__ fafb, int32_t n_sft, int32_t ncols,
                          int32_t n_pad, void* __restrict__ hi, void* __restrict__ lo) {
  const int64_t total = (int64_t)ncols * n_pad;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / n_pad;
    const int32_t a = (int32_t)(i - c * n_pad);
    const float x = a < n_sft ? fafb[c * n_sft + a] : 0.0f;
    if constexpr (BF16) {
      const uint32_t hp = pack_bf16(x, 0.0f);
      const float hx = __uint_as_float(hp << 16);
      const uint32_t lp = pack_bf16(x - hx, 0.0f);
      ((uint16_t*)hi)[i] = (uint16_t)(hp & 0xffffu);
      ((uint16_t*)lo)[i] = (uint16_t)(lp & 0xffffu);
    } else {
      const uint32_t hb = to_tf32(x);
      ((uint32_t*)hi)[i] = hb;
      ((uint32_t*)lo)[i] = to_tf32(x - __uint_as_float(hb));
    }
  }
}

}  // namespace tc

// ---------------------------------------------------------------- host -----

static int n_pad_of(int32_t n_sft) { return ((std::max(n_sft, 1) + 63) / 64) * 64; }
// N of the MMA: 4 columns per template, a multiple of 64 (the epilogue reads
// the accumulator 32 columns at a time per half).  Up to 48 templates one
// chunk of N <= 192; beyond, chunks of N = 128, which run two CTAs per SM
// (measured on the exp16 atoms: 64 templates 1.36 ms as two N = 128 chunks
// against 1.51 ms as one N = 256 chunk; 48 templates 1.25 ms as one N = 192
// chunk against 1.35 ms as two N = 128 chunks).
static int n_cols_of(int32_t T) {
  return T <= 48 ? ((4 * std::max(T, 1) + 63) / 64) * 64 : 128;
}

bool exp_tc_available(fmap_precision prec) { return prec == FMAP_TF32 || prec == FMAP_BF16X3; }

size_t exp_tc_operand_bytes(const fmap_grid&, int32_t n_sft, int32_t n_templates,
                            fmap_precision prec) {
  const size_t elem = prec == FMAP_BF16X3 ? 2 : 4;
  return 2 * elem * (size_t)4 * (size_t)std::max(n_templates, 1) * (size_t)n_pad_of(n_sft) + 256;
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

static cudaError_t encode_map(CUtensorMap* map, void* base, bool bf16, int32_t n_pad,
                              int32_t rows, int32_t box_rows) {
  auto enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)n_pad * (bf16 ? 2 : 4)};
  const cuuint32_t box[2] = {(cuuint32_t)(bf16 ? 64 : 32), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_exp_tc(fmap_plan_s* p, const fmap_atoms* a, float* d_2F, cudaStream_t s,
                          int64_t* tiles_used) {
  const fmap_grid& g = p->grid;
  const int64_t tiles = exp_tiles(g);
  *tiles_used = tiles;
  p->tiles = TileGeom{0, 1, tc::kRows, g.n_t0, (g.n_tau + tc::kRows - 1) / tc::kRows};
  if (tiles == 0 || p->n_templates == 0) return cudaSuccess;
  const bool bf16 = p->precision == FMAP_BF16X3;
  const int32_t T = p->n_templates;
  const int32_t n_pad = n_pad_of(p->n_sft);
  const int32_t ncols = 4 * T;
  const int N = n_cols_of(T);
  const size_t elem = bf16 ? 2 : 4;
  uint8_t* hi = (uint8_t*)p->ws.xop;
  uint8_t* lo = hi + (size_t)ncols * n_pad * elem;
  {
    const int64_t total = (int64_t)ncols * n_pad;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)p->n_sm * 8);
    if (bf16)
      tc::k_split_x<true><<<blocks, 256, 0, s>>>(a->fafb, p->n_sft, ncols, n_pad, hi, lo);
    else
      tc::k_split_x<false><<<blocks, 256, 0, s>>>(a->fafb, p->n_sft, ncols, n_pad, hi, lo);
    p->launches += 1;
  }
  if (!p->tmaps_ready) {
    cudaError_t e = encode_map((CUtensorMap*)p->tmap_hi, hi, bf16, n_pad, ncols, N);
    if (e == cudaSuccess) e = encode_map((CUtensorMap*)p->tmap_lo, lo, bf16, n_pad, ncols, N);
    if (e != cudaSuccess) return e;
    p->tmaps_ready = true;
  }
  tc::Params prm;
  prm.rel_t = p->ws.rel_t;
  prm.t_base = p->ws.t_base;
  prm.ax = plan_axes(p);
  prm.wtab = p->ws.wtab;
  prm.n_tab = p->n_tab;
  prm.g = g;
  prm.i0tab = p->ws.i0;
  prm.jend = p->ws.jend;
  prm.coef = p->ws.coef;
  prm.shared_antenna = a->shared_antenna;
  prm.n_templates = T;
  prm.n_cols = N;
  // TMEM: two accumulators of N columns, then the A stages.  Two stages where
  // that keeps a CTA within half the SM's TMEM columns (N = 64): two resident
  // CTAs run two MMA streams side by side; otherwise three stages where they
  // fit the SM's 512 columns (one CTA per SM), else two.
  const bool tab = g.window == FMAP_TABLE;
  const int acc_cols = 2 * N;
  int NS;
  if (!tab && acc_cols + 2 * tc::kAColsPerStage <= 256)
    NS = 2;
  else
    NS = acc_cols + 3 * tc::kAColsPerStage <= 512 ? 3 : 2;
  int tcols = 32;
  while (tcols < acc_cols + NS * tc::kAColsPerStage) tcols *= 2;
  if (tcols > 512) return cudaErrorInvalidConfiguration;
  prm.tmem_cols = tcols;
  prm.nblk = (g.n_tau + tc::kRows - 1) / tc::kRows;
  prm.map = d_2F;
  prm.parts = p->ws.partials;
  prm.stride = p->part_stride;
  prm.err = p->ws.dev_err;
  prm.wait_ns = (uint64_t)p->wait_ns;
  // shared memory: NS stages x (hi + lo) x N rows x 128 B, the staged times,
  // the table (TAB), the running sums (128 rows x N floats) and the 1 KB
  // alignment; at least enough to keep the resident CTAs within the 512
  // TMEM columns of an SM
  size_t smem = (size_t)NS * 2 * N * 128 + sizeof(float) * tc::kDtCap + 1024 +
                (tab ? sizeof(float2) * (kTabMax + 1) + 16 : 0) +
                (N == 64 ? 0 : (size_t)tc::kRows * N * 4);
  const size_t min_smem = tcols > 256 ? 120 * 1024 : 80 * 1024;
  smem = std::max(smem, min_smem);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  const int chunks = (ncols + N - 1) / N;
  dim3 grid((unsigned)tiles, (unsigned)chunks);
  const CUtensorMap* mh = (const CUtensorMap*)p->tmap_hi;
  const CUtensorMap* ml = (const CUtensorMap*)p->tmap_lo;
  cudaError_t err = cudaSuccess;
  auto run = [&](auto kern) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err == cudaSuccess) kern<<<grid, tc::kThreads, smem, s>>>(*mh, *ml, prm);
  };
  // N = 64 keeps the running sums in registers (the kernel's 2-CTA register
  // budget holds its 32 a thread), wider chunks in shared memory
  const bool rs = N == 64;
  if (bf16) {
    if (rs) {
      if (tab) run(tc::k_exp_tc<true, true, 3, true>);
      else run(tc::k_exp_tc<true, false, 2, true>);
    } else if (tab) {
      if (NS == 2) run(tc::k_exp_tc<true, true, 2, false>);
      else run(tc::k_exp_tc<true, true, 3, false>);
    } else if (NS == 2) {
      run(tc::k_exp_tc<true, false, 2, false>);
    } else {
      run(tc::k_exp_tc<true, false, 3, false>);
    }
  } else {
    if (rs) {
      if (tab) run(tc::k_exp_tc<false, true, 3, true>);
      else run(tc::k_exp_tc<false, false, 2, true>);
    } else if (tab) {
      if (NS == 2) run(tc::k_exp_tc<false, true, 2, false>);
      else run(tc::k_exp_tc<false, true, 3, false>);
    } else if (NS == 2) {
      run(tc::k_exp_tc<false, false, 2, false>);
    } else {
      run(tc::k_exp_tc<false, false, 3, false>);
    }
  }
  if (err != cudaSuccess) return err;
  p->launches += 1;
  return cudaGetLastError();
}

}  // namespace fmap
