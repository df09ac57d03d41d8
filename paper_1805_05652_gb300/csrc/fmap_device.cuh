// Device helpers shared by the F-map kernels: window index search, the 2F
// epilogue and the (max, argmax, log-sum-exp) partial reduction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fmap_internal.h"

namespace fmap {

constexpr int32_t kNoArg = 0x7fffffff;

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

__device__ __forceinline__ Partial partial_shfl_down(const Partial& p, int delta) {
  Partial q;
  q.max2F = __shfl_down_sync(0xffffffffu, p.max2F, delta);
  q.arg = __shfl_down_sync(0xffffffffu, p.arg, delta);
  q.sum = __shfl_down_sync(0xffffffffu, p.sum, delta);
  q.nvalid = __shfl_down_sync(0xffffffffu, p.nvalid, delta);
  return q;
}

__device__ __forceinline__ Partial partial_warp_reduce(Partial p) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) p = partial_merge(p, partial_shfl_down(p, d));
  return p;
}

// Block-wide reduction into lane 0 of warp 0; scratch holds >= nwarps entries.
// All threads of the block must call it.
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

// 2F from the sums of one template and the cell's coefficients.
__device__ __forceinline__ float two_f(const Coef& c, float fa_re, float fa_im, float fb_re,
                                       float fb_im) {
  const float e_re = fmaf(-c.beta, fa_re, fb_re);
  const float e_im = fmaf(-c.beta, fa_im, fb_im);
  const float fa2 = fmaf(fa_re, fa_re, fa_im * fa_im);
  const float e2 = fmaf(e_re, e_re, e_im * e_im);
  return fmaf(c.k1, fa2, c.k2 * e2);
}

// Coefficients from FP64 sums (D in FP64, the divisions in FP32).
__device__ __forceinline__ Coef make_coef(double A, double B, double C, int32_t count) {
  Coef c;
  const double D = A * B - C * C;
  if (count >= 2 && D > 0.0 && A > 0.0) {
    const float af = (float)A, cf = (float)C, df = (float)D;
    c.k1 = 2.0f / af;
    c.beta = cf / af;
    c.k2 = 2.0f * af / df;
    c.valid = (A * B > kCondThreshold * D) ? 2.0f : 1.0f;
  } else {
    c.k1 = 0.0f;
    c.beta = 0.0f;
    c.k2 = 0.0f;
    c.valid = 0.0f;
  }
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
