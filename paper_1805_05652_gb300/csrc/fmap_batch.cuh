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
  int32_t n_sft, T, shared, n_ant, groups, n_alloc, lanes;
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
  uint32_t* flag_bits;
  int32_t* n_flag;
  int64_t* flag_list;
  float4* pa;
  float4* perm_ant;
  float4* perm_x;
  int32_t* perm_gap;
  float4* rec_cells;
  TauTab* tauc;
  int64_t* ax;
  float4* px;
};

struct BUnits {
  const int64_t* offsets;   // [n_items + 1]
  int32_t n_items;
  int64_t total;
  unsigned long long* counter;
};

// Work of one unit in the phases whose natural unit is small (so that the
// per-unit claim and instance lookup stay a small share): rectangular
// coefficients in 256-entry blocks, index-table rows, fix-up slots.
constexpr int kCoefBlocksPerUnit = 8;
constexpr int kIdxRowsPerUnit = 8;
constexpr int kFixSlotsPerUnit = 4;
constexpr int kPermPerUnit = 4096;   // chunk-major copy entries per unit
constexpr int kBitsPerUnit = 4096;   // marked-entry bitmask words cleared per unit
static_assert(kFixSlots % kFixSlotsPerUnit == 0, "fix-up slot groups");

// Phases of the batch pipeline, in launch order.
enum BPhase {
  BP_PREP = 0,
  BP_INDEX,
  BP_EXP_PERM,
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

// A block claims units in increasing order, so the instance of its next
// unit is at or after that of its last one: thread 0 gallops forward from
// there (usually a step or two) and shares the result with the unit.
template <class F>
__device__ __forceinline__ void batch_loop(const BItem* __restrict__ items, const BUnits& u,
                                           F&& run) {
  __shared__ long long s_w;
  __shared__ int s_item;
  int last = 0;   // thread 0: instance of the previous unit
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const long long w = (long long)atomicAdd(u.counter, 1ull);
      s_w = w;
      if (w < u.total) {
        // last instance with offsets[i] <= w, searched in [last, n_items)
        int lo = last, step = 1;
        while (lo + step < u.n_items && u.offsets[lo + step] <= w) {
          lo += step;
          step <<= 1;
        }
        int hi = min(lo + step, u.n_items) - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (u.offsets[mid] <= w) lo = mid; else hi = mid - 1;
        }
        last = lo;
        s_item = lo;
      }
    }
    __syncthreads();
    const int64_t w = s_w;
    if (w >= u.total) return;
    const int i = s_item;
    run(items[i], w - u.offsets[i]);
  }
}

// Host launchers of the per-phase dispatchers (one per file holding the body).
cudaError_t launch_batch_phase(int phase, const BItem* d_items, const BUnits& u, int grid,
                               size_t dyn_smem, cudaStream_t s);
int batch_phase_threads(int phase);
const void* batch_phase_kernel(int phase);

}  // namespace fmap
