// fmap_marginalise_noalloc: the marginalisation of a given 2F map (max 2F,
// argmax, log Bayes factor) without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a
// latency-bound serving loop (cudaMalloc and cudaFree may synchronise the
// whole device and take milliseconds), or a host application that has handed
// all device memory to its own allocator and gives this library none.  For
// them this entry point keeps its scratch -- the per-tile reduction partials
// -- in a fixed array in the library's own device memory instead of a plan's
// workspace.
//
// The array is a file-scope __device__ object: every GPU that loads this
// library holds its kScratchBytes until the process exits.  Host code cannot
// use the array's name as a device address (in host code that name is a
// host-side stand-in), so the first call on each device, with that device
// current, looks its address up with cudaGetSymbolAddress and caches it with
// the context it belongs to; make that first call before any stream capture.
// A call in a different context (after cudaDeviceReset, which unloads the
// library's device code) looks the address up again, so make the first call
// after a reset outside stream capture too.  All calls share the one array:
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller.  Nothing in the
// array has to start at zero: each call writes every partial it later reads.
#include <cuda.h>

#include <mutex>
#include <string>

#include "fmap_internal.h"

namespace fmap {

constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB
constexpr int64_t kScratchPartials = (int64_t)(kScratchBytes / sizeof(Partial));
constexpr int kMaxDevices = 64;

static __device__ __align__(256) Partial g_scratch[kScratchPartials];

static std::mutex g_scratch_mu;
static Partial* g_scratch_ptr[kMaxDevices] = {};
static CUcontext g_scratch_ctx[kMaxDevices] = {};

// The driver's cuCtxGetCurrent, found through the runtime (the library does
// not link the driver directly, so it loads on machines without one).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
static CUcontext current_context() {
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)f;
  }
  CUcontext ctx = nullptr;
  if (!fn || fn(&ctx) != CUDA_SUCCESS) return nullptr;
  return ctx;
}

// Device address of g_scratch on the current device: looked up once per
// device and context (the context changes when the device is reset).
static fmap_status scratch_on_current_device(Partial** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal beyond the no-allocation scratch table");
    return FMAP_ERR_UNSUPPORTED;
  }
  // (null on a host thread the runtime has not used yet)
  CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev] || !ctx || g_scratch_ctx[dev] != ctx) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_scratch);   // (makes the device's context current)
    if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    ctx = current_context();
    g_scratch_ptr[dev] = (Partial*)ptr;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_ptr[dev];
  return FMAP_OK;
}

}  // namespace fmap

using namespace fmap;

extern "C" size_t fmap_noalloc_scratch_bytes(void) { return kScratchBytes; }

extern "C" fmap_status fmap_marginalise_noalloc(const fmap_grid* grid, int32_t n_templates,
                                                const float* d_2F, const uint8_t* d_valid,
                                                double log_prior_const, fmap_summary* d_summary,
                                                fmap_stream stream) {
  set_error("");
  std::string why;
  if (!grid_is_valid(grid, &why)) {
    set_error(why);
    return FMAP_ERR_ARG;
  }
  if (n_templates < 0 || n_templates > 65535) {
    set_error("n_templates must be in [0, 65535]");
    return FMAP_ERR_ARG;
  }
  const int64_t cells = (int64_t)grid->n_t0 * grid->n_tau;
  if (!d_summary || (cells > 0 && n_templates > 0 && !d_2F)) {
    set_error("map or summary pointer is NULL");
    return FMAP_ERR_ARG;
  }
  // per template: one 16-byte partial per 2048 cells, then the 32-byte results
  // of the first reduction level
  const int64_t tiles = marg_tiles(*grid);
  const int64_t need = (int64_t)n_templates * tiles * (int64_t)sizeof(Partial) + 32 +
                       (int64_t)n_templates * reduce_groups_of(tiles) * (int64_t)kGroupBytes;
  if (need > (int64_t)kScratchBytes) {
    set_error("map too large for the no-allocation scratch: needs " + std::to_string(need) +
              " bytes of reduction slots (16 bytes per template and 2048 cells), at most " +
              std::to_string(kScratchBytes) + " (8 MiB); use fmap_marginalise with a plan");
    return FMAP_ERR_ARG;
  }
  Partial* scratch = nullptr;
  fmap_status st = scratch_on_current_device(&scratch);
  if (st != FMAP_OK) return st;
  FMAP_CUDA(launch_marginalise_into(*grid, n_templates, d_2F, d_valid, scratch, log_prior_const,
                                    d_summary, (cudaStream_t)stream));
  return FMAP_OK;
}
