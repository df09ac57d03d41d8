// Kernels shared by both windows: input preparation, the window index tables
// (Eq. Fmn grid, window membership of Eq. winrect / winexp), the final
// per-template reduction and the standalone marginalisation.
#include <math.h>

#include "fmap_device.cuh"

namespace fmap {

// t -> t - t[0] as int32, with the data checks (strictly increasing,
// span < 2^31 s) latched into the plan's status word.
__global__ void k_prep(const int64_t* __restrict__ t, int32_t n, int32_t n_alloc,
                       int32_t* __restrict__ rel_t, int64_t* __restrict__ t_base,
                       uint32_t* __restrict__ err) {
  const int64_t base = t[0];
  for (int64_t i = n + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_alloc;
       i += (int64_t)gridDim.x * blockDim.x)
    rel_t[i] = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ti = t[i];
    const int64_t d = ti - base;
    uint32_t e = 0;
    if (d < 0 || d > 0x7fffffffLL - 1) e |= DEV_ERR_SPAN;
    if (i + 1 < n && t[i + 1] <= ti) e |= DEV_ERR_ORDER;
    if (e) atomicOr(err, e);
    rel_t[i] = (int32_t)(d & 0x7fffffffLL);
    if (i == 0) *t_base = base;
  }
}

// Window index tables: i0[m] = first atom with t >= t0_m; jend[m][n] = one
// past the last atom whose SFT ends by t0_m + L_n (L = tau or 3 tau),
// clamped to >= i0[m], so the window holds atoms [i0, jend).
__global__ void k_index(const int64_t* __restrict__ t, int32_t n_sft, fmap_grid g,
                        int32_t* __restrict__ i0tab, int32_t* __restrict__ jend) {
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  const int64_t lmul = (g.window == FMAP_RECT) ? 1 : 3;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < cells;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = c / g.n_tau, nn = c - m * g.n_tau;
    const int64_t t0 = g.t0_min + m * g.dt0;
    const int64_t tau = g.tau_min + nn * g.dtau;
    const int32_t i0 = lower_bound_i64(t, n_sft, t0);
    int32_t j = upper_bound_i64(t, n_sft, t0 + lmul * tau - g.t_sft);
    if (j < i0) j = i0;
    jend[c] = j;
    if (nn == 0) i0tab[m] = i0;
  }
}

cudaError_t launch_prep(fmap_plan_s* p, const int64_t* d_t, cudaStream_t s) {
  if (p->n_sft <= 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((p->n_sft + threads - 1) / threads, 4096);
  k_prep<<<blocks, threads, 0, s>>>(d_t, p->n_sft, rel_t_entries(p->n_sft), p->ws.rel_t,
                                    p->ws.t_base, p->ws.dev_err);
  p->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_index(fmap_plan_s* p, const int64_t* d_t, cudaStream_t s) {
  const int64_t cells = (int64_t)p->grid.n_t0 * p->grid.n_tau;
  if (cells == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t want = (cells + threads - 1) / threads;
  const int blocks = (int)std::min<int64_t>(want, (int64_t)p->n_sm * 16);
  k_index<<<blocks, threads, 0, s>>>(d_t, p->n_sft, p->grid, p->ws.i0, p->ws.jend);
  p->launches += 1;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Final reduction: one block per template over its tile partials, in FP64.
// Fixed per-thread order plus a fixed tree: the result is deterministic.
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;

__global__ void __launch_bounds__(kRedThreads)
k_final_reduce(const Partial* __restrict__ parts, int64_t n_tiles, int64_t fix0, int64_t n_fix,
               int64_t stride, int32_t n_tau, double log_prior, fmap_summary* __restrict__ out) {
  __shared__ float s_max[kRedThreads];
  __shared__ long long s_cnt[kRedThreads];
  __shared__ double s_sum[kRedThreads];
  __shared__ int32_t s_arg[kRedThreads];
  const int tid = threadIdx.x;
  const Partial* pp = parts + (int64_t)blockIdx.x * stride;
  float mx = -1.0f;
  long long cnt = 0;
  const int64_t n_all = n_tiles + n_fix;
  auto slot = [&](int64_t b) { return b < n_tiles ? pp[b] : pp[fix0 + (b - n_tiles)]; };
  for (int64_t b = tid; b < n_all; b += kRedThreads) {
    const Partial q = slot(b);
    if (q.nvalid > 0) {
      mx = fmaxf(mx, q.max2F);
      cnt += q.nvalid;
    }
  }
  s_max[tid] = mx;
  s_cnt[tid] = cnt;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (tid < w) {
      s_max[tid] = fmaxf(s_max[tid], s_max[tid + w]);
      s_cnt[tid] += s_cnt[tid + w];
    }
    __syncthreads();
  }
  const float M = s_max[0];
  const long long N = s_cnt[0];
  __syncthreads();
  double sum = 0.0;
  int32_t arg = kNoArg;
  if (N > 0) {
    for (int64_t b = tid; b < n_all; b += kRedThreads) {
      const Partial q = slot(b);
      if (q.nvalid > 0) {
        sum += (double)q.sum * exp(0.5 * ((double)q.max2F - (double)M));
        if (q.max2F == M && q.arg < arg) arg = q.arg;
      }
    }
  }
  s_sum[tid] = sum;
  s_arg[tid] = arg;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (tid < w) {
      s_sum[tid] += s_sum[tid + w];
      s_arg[tid] = min(s_arg[tid], s_arg[tid + w]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    fmap_summary r;
    r.reserved = 0;
    r.n_valid = N;
    if (N == 0) {
      r.max2F = 0.0f;
      r.m = -1;
      r.n = -1;
      r.logB = nan("");
    } else {
      r.max2F = M;
      r.m = s_arg[0] / n_tau;
      r.n = s_arg[0] % n_tau;
      r.logB = 0.5 * (double)M + log(s_sum[0]) - log((double)N) + log_prior;
    }
    out[blockIdx.x] = r;
  }
}

cudaError_t launch_final_reduce(fmap_plan_s* p, int64_t n_tiles, bool with_fix,
                                fmap_summary* d_summary, cudaStream_t s) {
  if (!d_summary || p->n_templates == 0) return cudaSuccess;
  const bool fix = with_fix && (int64_t)p->grid.n_t0 * p->grid.n_tau > 0;
  k_final_reduce<<<p->n_templates, kRedThreads, 0, s>>>(
      p->ws.partials, n_tiles, p->n_tiles, fix ? kFixSlots : 0, p->part_stride,
      p->grid.n_tau > 0 ? p->grid.n_tau : 1, p->log_prior, d_summary);
  p->launches += 1;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Standalone marginalisation of a given map: 2048 cells per tile.
// ---------------------------------------------------------------------------
constexpr int kMargThreads = 256;
constexpr int kMargPer = 8;

int64_t marg_tiles(const fmap_grid& g) {
  const int64_t cells = (int64_t)g.n_t0 * g.n_tau;
  return (cells + kMargThreads * kMargPer - 1) / (kMargThreads * kMargPer);
}

__global__ void __launch_bounds__(kMargThreads)
k_marg_partials(const float* __restrict__ map, const uint8_t* __restrict__ valid, int64_t cells,
                int64_t stride, Partial* __restrict__ parts) {
  __shared__ Partial scratch[kMargThreads / 32];
  const int64_t tile = blockIdx.x;
  const int64_t tmpl = blockIdx.y;
  const float* mp = map + tmpl * cells;
  const uint8_t* vp = valid ? valid + tmpl * cells : nullptr;
  Partial acc = partial_empty();
  const int64_t base = tile * (kMargThreads * kMargPer);
#pragma unroll
  for (int k = 0; k < kMargPer; ++k) {
    const int64_t c = base + k * kMargThreads + threadIdx.x;
    if (c < cells) {
      const bool ok = vp ? (vp[c] != 0) : true;
      partial_add(acc, mp[c], (int32_t)c, ok);
    }
  }
  acc = partial_block_reduce<kMargThreads / 32>(acc, scratch);
  if (threadIdx.x == 0) parts[tmpl * stride + tile] = acc;
}

cudaError_t launch_marginalise(fmap_plan_s* p, const float* d_2F, const uint8_t* d_valid,
                               fmap_summary* d_summary, cudaStream_t s) {
  const int64_t cells = (int64_t)p->grid.n_t0 * p->grid.n_tau;
  const int64_t tiles = marg_tiles(p->grid);
  if (tiles > 0 && p->n_templates > 0) {
    dim3 grid((unsigned)tiles, (unsigned)p->n_templates);
    k_marg_partials<<<grid, kMargThreads, 0, s>>>(d_2F, d_valid, cells, p->part_stride,
                                                  p->ws.partials);
    p->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_final_reduce(p, tiles, false, d_summary, s);
}

}  // namespace fmap
