// Persistent multi-instance launches (uneven batches).
//
// BItem describes one instance of a batch (its grid, atoms, outputs and the
// device pointers of its plan's workspace).  A phase of the batch pipeline is
// one launch of a dispatcher kernel over the work units of every instance:
// units of instance i are [offsets[i], offsets[i+1]); blocks pull units from
// an atomic counter and run the phase's device body with the instance's
// arguments and the unit as its block index.
#pragma once

#include "fmap_device.cuh"

namespace fmap {

struct BItem {
  fmap_grid g;
  int32_t n_sft, T, shared, n_ant, groups, n_alloc;
  int64_t cells, n_tiles, part_stride, red_groups, tiles_used, flag_entries;
  double log_prior;
  const int64_t* t;
  const float* antenna;
  const float* fafb;
  float* map;
  fmap_summary* summary;
  int32_t* rel_t;
  int64_t* t_base;
  uint32_t* dev_err;
  int32_t* i0;
  int32_t* jend;
  Coef* coef;
  Partial* partials;
  void* red_buf;
  int32_t* flag_blocks;
  int32_t* n_flag;
  int64_t* flag_list;
  double* pa;
  float4* px;
};

struct BUnits {
  const int64_t* offsets;   // [n_items + 1]
  int32_t n_items;
  int64_t total;
  unsigned long long* counter;
};

// Phases of the batch pipeline, in launch order.
enum BPhase {
  BP_PREP = 0,
  BP_INDEX,
  BP_RECT_ANT,
  BP_EXP_ANT,
  BP_RECT_COEF,
  BP_RECT_DATA,
  BP_EXP_REC,
  BP_RECT_CELLS,
  BP_FLAG_COUNT,
  BP_FLAG_SCAN,
  BP_FLAG_WRITE,
  BP_FIXUP,
  BP_RED_GROUPS,
  BP_RED_FINAL,
  BP_COUNT
};

template <class F>
__device__ __forceinline__ void batch_loop(const BItem* __restrict__ items, const BUnits& u,
                                           F&& run) {
  __shared__ long long s_w;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_w = (long long)atomicAdd(u.counter, 1ull);
    __syncthreads();
    const int64_t w = s_w;
    if (w >= u.total) return;
    int lo = 0, hi = u.n_items - 1;   // last instance with offsets[i] <= w
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (u.offsets[mid] <= w) lo = mid; else hi = mid - 1;
    }
    run(items[lo], w - u.offsets[lo]);
  }
}

// Host launchers of the per-phase dispatchers (one per file holding the body).
cudaError_t launch_batch_phase(int phase, const BItem* d_items, const BUnits& u, int grid,
                               size_t dyn_smem, cudaStream_t s);
int batch_phase_threads(int phase);
const void* batch_phase_kernel(int phase);

}  // namespace fmap
