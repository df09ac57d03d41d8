// Device helpers shared by the F-map kernels: window index search, the 2F
// epilogue and the (max, argmax, log-sum-exp) partial reduction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fmap_internal.h"

namespace fmap {

constexpr int32_t kNoArg = 0x7fffffff;

// ---- PTX helpers: shared-memory addresses, the global timer, mbarriers ----
// Every spin on an mbarrier is bounded by a limit in ns of %globaltimer: the
// plan's wait limit (kWaitNs by default), and kWaitNs for the drains that let
// copies already in flight land before a block that gave up exits.
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Non-blocking test of one phase (try_wait may suspend the thread for a
// hardware-defined time; a zero wait limit polls with this instead).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on one phase; false if it did not complete within limit_ns
// (0: give up when one non-blocking poll finds it incomplete).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitNs) {
  if (limit_ns == 0) return mbar_test_wait(bar, parity);
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > limit_ns) return false;
  return true;
}
// Bounded wait that also gives up at once when another block has already
// timed out (DEV_ERR_TIMEOUT set in *err), so a broken phase costs one
// timeout per launch, not one per block.  Sets the flag on its own timeout.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity,
                                                   uint32_t* err, uint64_t limit_ns = kWaitNs) {
  if (limit_ns == 0) {
    if (mbar_test_wait(bar, parity)) return true;
    atomicOr(err, DEV_ERR_TIMEOUT);
    return false;
  }
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (*(volatile uint32_t*)err & DEV_ERR_TIMEOUT) return false;
    if (globaltimer() - t0 > limit_ns) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      return false;
    }
    if (mbar_try_wait(bar, parity)) return true;
  }
}
// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of
// 16), completing `bytes` of transaction count on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- float-float (compensated FP32) arithmetic: a value is h + l with
// |l| <= ulp(h)/2, about 2^-44 relative after a chain of operations.  Built
// from the error-free transformations TwoSum (Knuth) and FMA-based TwoProd.
struct FF {
  float h, l;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = a.h * b.h;
  const float e = fmaf(a.h, b.h, -p);
  return fast_two_sum(p, e + fmaf(a.h, b.l, a.l * b.h));
}
__device__ __forceinline__ FF ff_mul_f(FF a, float b) {
  const float p = a.h * b;
  const float e = fmaf(a.h, b, -p);
  return fast_two_sum(p, fmaf(a.l, b, e));
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, s.l + a.l + b.l);
}
__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, FF{-b.h, -b.l}); }
// s <- s + w x: the product by FMA-based TwoProd, then a float-float addition
// (~2^-47 relative to the running sum per step).
__device__ __forceinline__ void ff_acc(FF& s, FF w, float x) {
  s = ff_add(s, ff_mul_f(w, x));
}
// s + r e with the product's low part folded into the sum's (no separate
// normalisation of r e): TwoProd of the high parts, TwoSum with s, one
// final renormalisation; ~2^-46 relative, as ff_add(s, ff_mul(r, e)).
__device__ __forceinline__ FF ff_fma_sum(FF s, FF r, FF e) {
  const float p = r.h * e.h;
  const float pe = fmaf(r.h, e.h, -p);
  const float t = s.h + p;
  const float bb = t - s.h;
  const float te = (s.h - (t - bb)) + (p - bb);
  return fast_two_sum(t, (s.l + fmaf(r.h, e.l, fmaf(r.l, e.h, pe))) + te);
}
// x + r e
__device__ __forceinline__ FF ff_axpy(FF r, FF e, float x) {
  const float p = r.h * e.h;
  const float pe = fmaf(r.h, e.h, -p);
  const FF s = two_sum(x, p);
  return fast_two_sum(s.h, s.l + pe + fmaf(r.h, e.l, r.l * e.h));
}
__device__ __forceinline__ FF ff_shfl_down(FF v, int d) {
  return {__shfl_down_sync(0xffffffffu, v.h, d), __shfl_down_sync(0xffffffffu, v.l, d)};
}
__device__ __forceinline__ FF ff_of(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

// Fills the per-tau constants of one tau value (one thread).  The one-SFT decay is
// an FP64 exp split into a float pair; its powers come by binary powering in
// float-float (~k ulp of 2^-48).
__device__ __forceinline__ void tau_tab_fill(const fmap_grid& g, int64_t tau, TauTab* out) {
  TauTab t;
  t.inv_tau = 1.0 / (double)tau;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const double inv_s = (double)(s + 1) * t.inv_tau;
    t.c2[s] = (float)(-1.4426950408889634 * inv_s);
    const FF rho1 = ff_of(exp(-(double)g.t_sft * inv_s));
    for (int k = 0; k < kPowTab; ++k) {
      FF acc{1.0f, 0.0f}, r = rho1;
      for (int q = k; q; q >>= 1) {
        if (q & 1) acc = ff_mul(acc, r);
        r = ff_mul(r, r);
      }
      t.pw[s][k] = make_float2(acc.h, acc.l);
    }
  }
  *out = t;
}
// Decay over one gap between consecutive atoms: a table entry (pw of the
// tau's TauTab) for gaps of 1..kPowTab-1 whole SFTs, FP64 exp otherwise
// (gaps off the T_sft lattice; inv_s = s / tau).
__device__ __forceinline__ FF gap_decay(int32_t gap, int32_t t_sft, float inv_tsft,
                                        const float2* __restrict__ tab, double inv_s) {
  const int32_t k = __float2int_rn((float)gap * inv_tsft);
  if (k >= 1 && k < kPowTab && k * t_sft == gap) {
    const float2 v = tab[k];
    return {v.x, v.y};
  }
  return ff_of(exp(-(double)gap * inv_s));
}

// Generic window w(x) from its table (entries k = 0..n-1: (w_k, w_{k+1} -
// w_k), then the sentinel (0, 0)): linear between samples, 0 past the last.
// u = x (n - 1) / X is the position in sample units (u >= 0).
__device__ __forceinline__ float tab_weight(float u, const float2* tab, int32_t n) {
  const int32_t k = min(__float2int_rz(u), n);   // u beyond the table: the sentinel
  const float2 e = tab[k];
  return fmaf(u - (float)k, e.y, e.x);
}
__device__ __forceinline__ double tab_weight64(double u, const float2* tab, int32_t n) {
  const double fk = floor(u);
  const int32_t k = fk >= (double)n ? n : (int32_t)fk;
  const float2 e = tab[k];
  return (double)e.x + (u - (double)k) * (double)e.y;
}
// Sample units per second of (t - t0) for a tau: (n - 1) / (X tau), X = c / 8.
__host__ __device__ __forceinline__ double tab_scale(int32_t n, int32_t cut8, int64_t tau) {
  return (double)(n - 1) * 8.0 / ((double)cut8 * (double)tau);
}

// Compensated recurrence E <- x + r E (Horner's rule with error-free
// transformations, after Graillat, Langlois and Louvet's compensated Horner
// scheme): E = h + c with h the plain FP32 recurrence and c carrying its
// rounding errors (the TwoProd error of r.h h, the TwoSum error of adding x,
// and the low part r.l of the decay).  The pair is left unnormalised between
// calls; ch_norm folds c back into h.
__device__ __forceinline__ void ch_step(FF r, float x, float& h, float& c) {
  const float p = r.h * h;
  const float pe = fmaf(r.h, h, -p);
  const float s = p + x;
  const float bb = s - p;
  const float se = (p - (s - bb)) + (x - bb);
  c = fmaf(r.h, c, fmaf(r.l, h, pe + se));
  h = s;
}
// R <- r R for the compensated running product of the decays.
__device__ __forceinline__ void ch_mul(FF r, float& h, float& c) {
  const float p = r.h * h;
  const float pe = fmaf(r.h, h, -p);
  c = fmaf(r.h, c, fmaf(r.l, h, pe));
  h = p;
}
__device__ __forceinline__ void ch_norm(float& h, float& c) {
  const float s = h + c;
  c = c - (s - h);
  h = s;
}

__device__ __forceinline__ Partial partial_empty() {
  Partial p;
  p.max2F = -1.0f;
  p.arg = kNoArg;
  p.sum = 0.0f;
  p.nvalid = 0;
  return p;
}

// Merge two partials (max 2F, lowest argmax on ties, rescaled exp-sum).
__device__ __forceinline__ Partial partial_merge(const Partial& a, const Partial& b) {
  if (a.nvalid == 0) return b;
  if (b.nvalid == 0) return a;
  Partial r;
  if (a.max2F > b.max2F) {
    r.max2F = a.max2F;
    r.arg = a.arg;
    r.sum = a.sum + b.sum * __expf(0.5f * (b.max2F - a.max2F));
  } else if (b.max2F > a.max2F) {
    r.max2F = b.max2F;
    r.arg = b.arg;
    r.sum = b.sum + a.sum * __expf(0.5f * (a.max2F - b.max2F));
  } else {
    r.max2F = a.max2F;
    r.arg = min(a.arg, b.arg);
    r.sum = a.sum + b.sum;
  }
  r.nvalid = a.nvalid + b.nvalid;
  return r;
}

// Add one cell to a running partial.
__device__ __forceinline__ void partial_add(Partial& p, float twoF, int32_t idx, bool valid) {
  if (!valid) return;
  if (p.nvalid == 0) {
    p.max2F = twoF;
    p.arg = idx;
    p.sum = 1.0f;
    p.nvalid = 1;
    return;
  }
  if (twoF > p.max2F) {
    p.sum = p.sum * __expf(0.5f * (p.max2F - twoF)) + 1.0f;
    p.max2F = twoF;
    p.arg = idx;
  } else {
    p.sum += __expf(0.5f * (twoF - p.max2F));
    if (twoF == p.max2F && idx < p.arg) p.arg = idx;
  }
  p.nvalid += 1;
}

// Warp-wide merge (all 32 lanes; the result in every lane).  2F >= 0, so a
// valid partial's maximum orders like its bit pattern: the warp maximum is
// one integer max reduction, each lane rescales its sum to it (one exp),
// the sums add in a fixed butterfly order, and the lowest index among the
// lanes at the maximum and the valid count are integer reductions.
__device__ __forceinline__ Partial partial_warp_reduce(Partial p) {
  const bool has = p.nvalid > 0;
  const unsigned mu = __reduce_max_sync(0xffffffffu, has ? __float_as_uint(p.max2F) + 1u : 0u);
  if (mu == 0u) return partial_empty();
  const float M = __uint_as_float(mu - 1u);
  float s = has ? p.sum * __expf(0.5f * (p.max2F - M)) : 0.0f;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  Partial r;
  r.max2F = M;
  r.arg = (int32_t)__reduce_min_sync(0xffffffffu,
                                     has && p.max2F == M ? (unsigned)p.arg : (unsigned)kNoArg);
  r.sum = s;
  r.nvalid = (int32_t)__reduce_add_sync(0xffffffffu, (unsigned)p.nvalid);
  return r;
}

// Block-wide reduction into lane 0 of warp 0 (warp partials merged by warp
// 0); scratch holds >= nwarps entries.  All threads of the block must call it.
template <int NWARPS>
__device__ __forceinline__ Partial partial_block_reduce(Partial p, Partial* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  p = partial_warp_reduce(p);
  if (lane == 0) scratch[warp] = p;
  __syncthreads();
  Partial r = partial_empty();
  if (warp == 0) {
    r = lane < NWARPS ? scratch[lane] : partial_empty();
    r = partial_warp_reduce(r);
  }
  __syncthreads();
  return r;
}

// The same over consecutive calls of one loop with a single barrier:
// scratch holds 2 x NWARPS entries, used alternately by parity, so a call's
// warp partials never overwrite those warp 0 may still read from the call
// before (the barrier of the call in between orders them).
template <int NWARPS>
__device__ __forceinline__ Partial partial_block_reduce_alt(Partial p, Partial* scratch,
                                                            int parity) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Partial* sc = scratch + (parity & 1) * NWARPS;
  p = partial_warp_reduce(p);
  if (lane == 0) sc[warp] = p;
  __syncthreads();
  Partial r = partial_empty();
  if (warp == 0) {
    r = lane < NWARPS ? sc[lane] : partial_empty();
    r = partial_warp_reduce(r);
  }
  return r;
}

// 2F from the sums of one template and the cell's coefficients.
__device__ __forceinline__ float two_f(const Coef& c, float fa_re, float fa_im, float fb_re,
                                       float fb_im) {
  const float e_re = fmaf(-c.beta, fa_re, fb_re);
  const float e_im = fmaf(-c.beta, fa_im, fb_im);
  const float fa2 = fmaf(fa_re, fa_re, fa_im * fa_im);
  const float e2 = fmaf(e_re, e_re, e_im * e_im);
  return fmaf(c.k1, fa2, c.k2 * e2);
}

// Stores the coefficients of entry e and marks it in the bitmask of the
// ill-conditioned entries when it goes to the fix-up (valid == 2).
__device__ __forceinline__ void store_coef(Coef* __restrict__ coef, uint32_t* __restrict__ bits,
                                           int64_t e, const Coef& c) {
  coef[e] = c;
  if (c.valid == 2.0f) atomicOr(bits + (e >> 5), 1u << (uint32_t)(e & 31));
}

// Coefficients from float-float sums: D = AB - C^2 from exact FMA products
// (relative error ~2^-44 AB, so ~1e-11 of D for AB/D <= 100); the
// divisions in FP32.  A cell whose D is not clearly positive or whose
// AB/D > 100 goes to the fix-up, which decides its validity from
// float-float sums of the window.
__device__ __forceinline__ Coef make_coef_ff(FF A, FF B, FF C, int32_t count) {
  Coef c{0.0f, 0.0f, 0.0f, 0.0f};
  if (count < 2) return c;
  const FF D = ff_sub(ff_mul(A, B), ff_mul(C, C));
  const float af = A.h, cf = C.h, df = D.h;
  if (!(af > 0.0f)) {
    c.valid = 2.0f;
    return c;
  }
  // two correctly rounded reciprocals instead of three divisions (k1 is
  // exact as before; beta and k2 within 1.5 ulp)
  const float ia = __frcp_rn(af);
  c.k1 = 2.0f * ia;
  c.beta = cf * ia;
  c.k2 = (2.0f * af) * __frcp_rn(df);
  // A B > 100 D, compared in float-float
  const FF ab = ff_mul(A, B), d100 = ff_mul_f(D, kCondThreshold);
  const FF gap = ff_sub(d100, ab);
  c.valid = (df > 0.0f && gap.h + gap.l >= 0.0f) ? 1.0f : 2.0f;
  return c;
}

// First index with t[i] > x (x as int64), over n entries of int64 times.
__device__ __forceinline__ int32_t upper_bound_i64(const int64_t* t, int32_t n, int64_t x) {
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (t[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// First index with t[i] >= x.
__device__ __forceinline__ int32_t lower_bound_i64(const int64_t* t, int32_t n, int64_t x) {
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (t[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

}  // namespace fmap
