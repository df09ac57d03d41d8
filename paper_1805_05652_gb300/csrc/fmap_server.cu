// Serving loop: F-map requests admitted by device memory and run with
// continuous batching.
//
// A request (one grid, its atoms, 1..T templates) is copied at submission into
// a pinned host arena.  A worker thread admits queued requests in arrival
// order while a stream slot is free and the request's device footprint (plan
// workspace + atoms + outputs) fits in the device pool, which is allocated
// once at creation and sub-allocated per request (no cudaMalloc per request).
// Each admitted request runs on its own stream -- upload, the plan's compute,
// download -- so requests that arrive while others are on the GPU overlap
// with them.  The worker retires finished requests by their events, returns
// their memory and wakes fmap_poll callers.  A request's results do not
// depend on what else is in flight: it has its own plan and workspace, and
// the kernels' tiling and reduction order depend only on its own sizes.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fmap_internal.h"

namespace fmap {

// First-fit allocator over [0, size) with coalescing frees.
class RangeAllocator {
 public:
  explicit RangeAllocator(size_t size = 0) { reset(size); }
  void reset(size_t size) {
    free_.clear();
    size_ = size;
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t capacity() const { return size_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0;
};

struct Request {
  uint64_t ticket = 0;
  fmap_grid grid{};
  int32_t n_sft = 0, T = 0, shared = 1;
  bool want_map = false;
  // pinned host arena region: inputs then outputs
  size_t pin_off = 0, pin_bytes = 0;
  int64_t* h_t = nullptr;
  float* h_ant = nullptr;
  float* h_x = nullptr;
  fmap_summary* h_sum = nullptr;
  uint32_t* h_err = nullptr;       // the plan's device status word, copied back
  float* h_map = nullptr;
  // device pool region
  size_t dev_off = 0, dev_bytes = 0, ws_bytes = 0;
  fmap_plan_s* plan = nullptr;
  fmap_precision prec = FMAP_FP64;   // the plan's precision and flags
  uint32_t pflags = 0;
  bool urgent = false;               // runs on the slot's high-priority stream
  cudaStream_t stream = nullptr;
  int slot = -1;
  enum { QUEUED, RUNNING, DONE } state = QUEUED;
  fmap_status status = FMAP_OK;
  std::string error;
  int64_t t_submit_ns = 0, t_done_ns = 0;
};

static int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace fmap

struct fmap_server_s {
  fmap_server_config cfg{};
  int device = 0;
  char* dev_pool = nullptr;
  char* pin_pool = nullptr;
  fmap::RangeAllocator dev_alloc, pin_alloc;
  std::vector<cudaStream_t> streams;    // per slot: normal priority
  std::vector<cudaStream_t> ustreams;   // per slot: high priority (small requests)
  std::vector<cudaEvent_t> events;
  std::vector<fmap::Request*> slots;   // running request per stream slot
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<fmap::Request*> queue;
  std::unordered_map<uint64_t, fmap::Request*> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  int64_t completed = 0;
  int64_t peak_running = 0;
};

namespace fmap {

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Estimated GPU milliseconds of a request, in the form of App. A's timing
// model (per template: a term in the atoms scanned, one in the windowed
// sums N_sums and one in the cells N_t0 N_tau, plus a constant), with the
// constants fitted on GB300 to the serving mix (summaries refined; median
// error ~20 %).  Used only to choose between the exponential forms and the
// stream priority: a poor estimate costs speed, never accuracy.
struct CostModel {
  // N_sums of an exponential / rectangular grid, from a 64 x 64 sample of
  // its cells: a window holds min(L, data end - max(t0, first atom)) of the
  // data span, at the data set's mean atom density.
  static double n_sums(const fmap_grid& g, const int64_t* t, int32_t n) {
    if (n <= 0 || g.n_t0 <= 0 || g.n_tau <= 0) return 0.0;
    const double first = (double)t[0], end = (double)t[n - 1] + (double)g.t_sft;
    const double density = (double)n / ((end - first) / (double)g.t_sft);
    const int km = std::min<int32_t>(g.n_t0, 64), kn = std::min<int32_t>(g.n_tau, 64);
    double acc = 0.0;
    for (int a = 0; a < km; ++a) {
      const int64_t m = (int64_t)(g.n_t0 - 1) * a / std::max(km - 1, 1);
      const double t0 = (double)(g.t0_min + m * g.dt0);
      const double room = std::max(0.0, end - std::max(t0, first));
      for (int b = 0; b < kn; ++b) {
        const int64_t nn = (int64_t)(g.n_tau - 1) * b / std::max(kn - 1, 1);
        const double L = (double)window_len(g, g.tau_min + nn * g.dtau);
        acc += std::min(L, room) / (double)g.t_sft * density;
      }
    }
    return acc / ((double)km * kn) * (double)g.n_t0 * (double)g.n_tau;
  }
  static double rect_ms(const fmap_grid& g, int32_t n, int32_t T) {
    return 3.48e-9 * T * (double)g.n_t0 * g.n_tau + 5.78e-7 * T * (double)n + 0.29;
  }
  static double exp_tc_ms(const fmap_grid& g, double sums, int32_t T) {
    return 3.98e-11 * T * sums + 1.58e-8 * T * (double)g.n_t0 * g.n_tau + 0.85;
  }
  static double exp_rec_ms(const fmap_grid& g, int32_t n, int32_t T) {
    return 8.25e-9 * T * (double)g.n_tau * n + 1.21e-8 * T * (double)g.n_t0 * g.n_tau +
           5.85e-6 * T * (double)g.n_tau + 0.30;
  }
};
constexpr double kUrgentMs = 1.0;

// Bytes of a request's inputs and outputs.  The device always holds the map
// (the refinement of the summaries reads and rewrites it); the pinned host
// arena holds it only when the request asked for it.
static void request_sizes(const Request& r, size_t* in_bytes, size_t* out_bytes,
                          size_t* host_out_bytes) {
  const size_t n = (size_t)r.n_sft, T = (size_t)r.T;
  const size_t cells = (size_t)r.grid.n_t0 * (size_t)r.grid.n_tau;
  *in_bytes = align256(8 * n) + align256(4 * 3 * n * (r.shared ? 1 : T)) + align256(4 * 4 * n * T);
  const size_t sums = align256(sizeof(fmap_summary) * T) + 256;
  *out_bytes = sums + align256(4 * cells * T);
  *host_out_bytes = sums + (r.want_map ? align256(4 * cells * T) : 0);
}

// Launch one admitted request on its slot's stream (lock held).
static fmap_status launch_request(fmap_server_s* s, Request* r) {
  size_t in_b, out_b, hout_b;
  request_sizes(*r, &in_b, &out_b, &hout_b);
  char* d = s->dev_pool + r->dev_off;
  r->plan = new (std::nothrow) fmap_plan_s();
  if (!r->plan) return FMAP_ERR_NOMEM;
  fmap_status st = plan_init(r->plan, &r->grid, r->n_sft, r->T, r->prec, r->pflags, d, r->ws_bytes);
  if (st != FMAP_OK) return st;
  char* q = d + align256(r->ws_bytes);
  const size_t n = (size_t)r->n_sft, T = (size_t)r->T;
  int64_t* d_t = (int64_t*)q;
  q += align256(8 * n);
  float* d_ant = (float*)q;
  q += align256(4 * 3 * n * (r->shared ? 1 : T));
  float* d_x = (float*)q;
  q += align256(4 * 4 * n * T);
  fmap_summary* d_sum = (fmap_summary*)q;
  q += align256(sizeof(fmap_summary) * T) + 256;
  float* d_map = (float*)q;
  cudaStream_t st_ = r->urgent ? s->ustreams[r->slot] : s->streams[r->slot];
  r->stream = st_;
  const size_t cells = (size_t)r->grid.n_t0 * (size_t)r->grid.n_tau;
  if (n > 0) {
    FMAP_CUDA(cudaMemcpyAsync(d_t, r->h_t, 8 * n, cudaMemcpyHostToDevice, st_));
    FMAP_CUDA(cudaMemcpyAsync(d_ant, r->h_ant, 4 * 3 * n * (r->shared ? 1 : T),
                              cudaMemcpyHostToDevice, st_));
    if (T > 0) FMAP_CUDA(cudaMemcpyAsync(d_x, r->h_x, 4 * 4 * n * T, cudaMemcpyHostToDevice, st_));
  }
  fmap_atoms a{r->n_sft, r->T, r->shared, d_t, d_ant, d_x};
  st = r->grid.window == FMAP_RECT
           ? fmap_compute_rect(r->plan, &a, d_map, d_sum, (fmap_stream)st_)
           : fmap_compute_exp(r->plan, &a, d_map, d_sum, (fmap_stream)st_);
  if (st != FMAP_OK) return st;
  if (T > 0)
    FMAP_CUDA(cudaMemcpyAsync(r->h_sum, d_sum, sizeof(fmap_summary) * T, cudaMemcpyDeviceToHost,
                              st_));
  if (r->want_map && cells * T > 0)
    FMAP_CUDA(cudaMemcpyAsync(r->h_map, d_map, 4 * cells * T, cudaMemcpyDeviceToHost, st_));
  FMAP_CUDA(cudaMemcpyAsync(r->h_err, r->plan->ws.dev_err, sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, st_));
  FMAP_CUDA(cudaEventRecord(s->events[r->slot], st_));
  return FMAP_OK;
}

static void finish_request(fmap_server_s* s, Request* r, fmap_status st, const std::string& err) {
  if (r->plan) {
    plan_release(r->plan);
    delete r->plan;
    r->plan = nullptr;
  }
  if (r->dev_bytes) s->dev_alloc.release(r->dev_off, r->dev_bytes);
  r->dev_bytes = 0;
  if (r->slot >= 0) s->slots[r->slot] = nullptr;
  r->slot = -1;
  r->status = st;
  r->error = err;
  r->state = Request::DONE;
  r->t_done_ns = now_ns();
  s->completed += 1;
}

static void worker_loop(fmap_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progress = false;
    // retire finished requests
    for (size_t k = 0; k < s->slots.size(); ++k) {
      Request* r = s->slots[k];
      if (!r) continue;
      const cudaError_t q = cudaEventQuery(s->events[k]);
      if (q == cudaErrorNotReady) continue;
      fmap_status st = FMAP_OK;
      std::string err;
      if (q != cudaSuccess) {
        st = FMAP_ERR_CUDA;
        err = cudaGetErrorString(q);
      } else if (*r->h_err) {
        st = dev_err_status(*r->h_err);
        err = dev_err_message(*r->h_err);
      }
      finish_request(s, r, st, err);
      progress = true;
    }
    if (progress) s->cv_done.notify_all();
    // admit in arrival order while a slot and device memory are free
    while (!s->queue.empty()) {
      int slot = -1;
      for (size_t k = 0; k < s->slots.size(); ++k)
        if (!s->slots[k]) {
          slot = (int)k;
          break;
        }
      if (slot < 0) break;
      Request* r = s->queue.front();
      size_t off = 0;
      if (!s->dev_alloc.alloc(r->dev_bytes, &off)) break;   // wait for memory to free up
      s->queue.pop_front();
      r->dev_off = off;
      r->slot = slot;
      s->slots[slot] = r;
      r->state = Request::RUNNING;
      int64_t run = 0;
      for (auto* q : s->slots) run += q != nullptr;
      s->peak_running = std::max(s->peak_running, run);
      const fmap_status st = launch_request(s, r);
      if (st != FMAP_OK) {
        // copies and kernels queued before the failure may still be writing
        // the request's device range: let them finish before it is reused
        const std::string why = fmap_last_error();
        cudaStreamSynchronize(r->stream ? r->stream : s->streams[slot]);
        cudaGetLastError();
        finish_request(s, r, st, why);
      }
      progress = true;
    }
    if (progress) {
      s->cv_done.notify_all();
      continue;
    }
    bool running = false;
    for (auto* r : s->slots) running |= (r != nullptr);
    s->cv_work.wait_for(lk, std::chrono::microseconds(running ? 20 : 2000));
  }
}

}  // namespace fmap

using namespace fmap;

extern "C" {

fmap_status fmap_server_create(fmap_server_t** out, const fmap_server_config* cfg) {
  set_error("");
  if (!out || !cfg) {
    set_error("NULL argument");
    return FMAP_ERR_ARG;
  }
  *out = nullptr;
  if (cfg->max_inflight < 1 || cfg->max_inflight > 64 || cfg->device_mem_budget < (1u << 20) ||
      cfg->pinned_bytes < (1u << 20) || cfg->exp_mode > FMAP_SERVER_EXP_AUTO) {
    set_error("max_inflight must be in [1, 64]; device and pinned budgets >= 1 MiB; "
              "exp_mode FMAP_SERVER_EXP_*");
    return FMAP_ERR_ARG;
  }
  fmap_server_s* s = new (std::nothrow) fmap_server_s();
  if (!s) return FMAP_ERR_NOMEM;
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  cudaError_t e = cudaMalloc((void**)&s->dev_pool, cfg->device_mem_budget);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->pin_pool, cfg->pinned_bytes, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->dev_pool);
    delete s;
    set_error("server pool allocation failed");
    return FMAP_ERR_NOMEM;
  }
  s->dev_alloc.reset(cfg->device_mem_budget);
  s->pin_alloc.reset(cfg->pinned_bytes);
  s->streams.resize(cfg->max_inflight);
  s->ustreams.resize(cfg->max_inflight);
  s->events.resize(cfg->max_inflight);
  s->slots.assign(cfg->max_inflight, nullptr);
  int lo_prio = 0, hi_prio = 0;   // (numerically lower = higher priority)
  cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
  for (int k = 0; k < cfg->max_inflight; ++k) {
    cudaStreamCreateWithPriority(&s->streams[k], cudaStreamNonBlocking, lo_prio);
    cudaStreamCreateWithPriority(&s->ustreams[k], cudaStreamNonBlocking, hi_prio);
    cudaEventCreateWithFlags(&s->events[k], cudaEventDisableTiming);
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return FMAP_OK;
}

void fmap_server_destroy(fmap_server_t* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto st : s->streams) cudaStreamSynchronize(st);
  for (auto st : s->ustreams) cudaStreamSynchronize(st);
  for (auto& kv : s->all) {
    Request* r = kv.second;
    if (r->plan) {
      plan_release(r->plan);
      delete r->plan;
    }
    delete r;
  }
  for (auto st : s->streams) cudaStreamDestroy(st);
  for (auto st : s->ustreams) cudaStreamDestroy(st);
  for (auto ev : s->events) cudaEventDestroy(ev);
  cudaFree(s->dev_pool);
  cudaFreeHost(s->pin_pool);
  delete s;
}

fmap_status fmap_submit(fmap_server_t* s, const fmap_grid* grid, const fmap_atoms* h,
                        uint32_t flags, uint64_t* ticket) {
  set_error("");
  if (!s || !grid || !h || !ticket) {
    set_error("NULL argument");
    return FMAP_ERR_ARG;
  }
  if (flags & ~(uint32_t)FMAP_SUBMIT_MAP) {
    set_error("unknown submit flags");
    return FMAP_ERR_ARG;
  }
  Request* r = new (std::nothrow) Request();
  if (!r) return FMAP_ERR_NOMEM;
  r->grid = *grid;
  r->n_sft = h->n_sft;
  r->T = h->n_templates;
  r->shared = h->shared_antenna ? 1 : 0;
  r->want_map = (flags & FMAP_SUBMIT_MAP) != 0;
  if (r->n_sft < 0 || r->T < 0 || r->T > 65535 ||
      (r->n_sft > 0 && (!h->t || !h->antenna || (r->T > 0 && !h->fafb)))) {
    delete r;
    set_error("bad atoms");
    return FMAP_ERR_ARG;
  }
  if (grid->window == FMAP_TABLE) {
    delete r;
    set_error("table windows are not served");
    return FMAP_ERR_ARG;
  }
  // the form of the request, and its priority, by the cost model
  r->pflags = r->shared ? 0u : (uint32_t)FMAP_PLAN_PER_TEMPLATE_ANTENNA;
  double est = 0.0;
  if (grid->window == FMAP_RECT) {
    r->prec = s->cfg.rect_precision;
    est = CostModel::rect_ms(*grid, r->n_sft, r->T);
  } else {
    // (data sets past the recurrence's shared-memory limit take exp_precision)
    const bool rec_ok = exp_rec_supported(r->n_sft, grid->n_t0);
    const double rec = CostModel::exp_rec_ms(*grid, r->n_sft, r->T);
    bool use_rec = rec_ok && s->cfg.exp_mode == FMAP_SERVER_EXP_RECURRENCE;
    double other = rec;
    if (!use_rec) {
      const double sums = r->n_sft > 0 ? CostModel::n_sums(*grid, h->t, r->n_sft) : 0.0;
      other = CostModel::exp_tc_ms(*grid, sums, r->T);
      use_rec = rec_ok && s->cfg.exp_mode == FMAP_SERVER_EXP_AUTO && rec < other;
    }
    r->prec = use_rec ? FMAP_FP64 : s->cfg.exp_precision;
    if (use_rec) r->pflags |= (uint32_t)FMAP_PLAN_EXP_RECURRENCE;
    est = use_rec ? rec : other;
  }
  r->urgent = est < kUrgentMs;
  fmap_status st = plan_footprint(grid, r->n_sft, r->T, r->prec, r->pflags, &r->ws_bytes);
  if (st != FMAP_OK) {
    delete r;
    return st;
  }
  size_t in_b, out_b, hout_b;
  request_sizes(*r, &in_b, &out_b, &hout_b);
  r->dev_bytes = align256(r->ws_bytes) + in_b + out_b;
  r->pin_bytes = in_b + hout_b;
  if (r->dev_bytes > s->dev_alloc.capacity()) {
    delete r;
    set_error("request larger than the server's device memory budget");
    return FMAP_ERR_NOMEM;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  if (!s->pin_alloc.alloc(r->pin_bytes, &r->pin_off)) {
    delete r;
    set_error("pinned staging full: poll finished requests, then resubmit");
    return FMAP_ERR_BUSY;
  }
  char* pbase = s->pin_pool + r->pin_off;
  const size_t n = (size_t)r->n_sft, T = (size_t)r->T;
  r->h_t = (int64_t*)pbase;
  pbase += align256(8 * n);
  r->h_ant = (float*)pbase;
  pbase += align256(4 * 3 * n * (r->shared ? 1 : T));
  r->h_x = (float*)pbase;
  pbase += align256(4 * 4 * n * T);
  r->h_sum = (fmap_summary*)pbase;
  pbase += align256(sizeof(fmap_summary) * T);
  r->h_err = (uint32_t*)pbase;
  pbase += 256;
  r->h_map = r->want_map ? (float*)pbase : nullptr;
  lk.unlock();
  if (n > 0) {
    std::memcpy(r->h_t, h->t, 8 * n);
    std::memcpy(r->h_ant, h->antenna, 4 * 3 * n * (r->shared ? 1 : T));
    if (T > 0) std::memcpy(r->h_x, h->fafb, 4 * 4 * n * T);
  }
  lk.lock();
  r->ticket = s->next_ticket++;
  r->t_submit_ns = now_ns();
  s->all[r->ticket] = r;
  s->queue.push_back(r);
  *ticket = r->ticket;
  lk.unlock();
  s->cv_work.notify_all();
  return FMAP_OK;
}

fmap_status fmap_poll(fmap_server_t* s, uint64_t ticket, fmap_summary* h_summary, float* h_2F,
                      int64_t wait_us) {
  set_error("");
  if (!s) {
    set_error("server is NULL");
    return FMAP_ERR_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) {
    set_error("unknown ticket");
    return FMAP_ERR_BUSY;
  }
  Request* r = it->second;
  if (r->state != Request::DONE && wait_us != 0) {
    auto pred = [&] { return r->state == Request::DONE; };
    if (wait_us < 0)
      s->cv_done.wait(lk, pred);
    else
      s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), pred);
  }
  if (r->state != Request::DONE) return FMAP_PENDING;
  const fmap_status st = r->status;
  if (st == FMAP_OK) {
    const size_t T = (size_t)r->T;
    const size_t cells = (size_t)r->grid.n_t0 * (size_t)r->grid.n_tau;
    if (h_summary && T) std::memcpy(h_summary, r->h_sum, sizeof(fmap_summary) * T);
    if (h_2F && r->want_map && T * cells) std::memcpy(h_2F, r->h_map, 4 * cells * T);
  } else {
    set_error(r->error);
  }
  s->pin_alloc.release(r->pin_off, r->pin_bytes);
  s->all.erase(it);
  delete r;
  return st;
}

fmap_status fmap_server_peak(fmap_server_t* s, int64_t* peak_running) {
  if (!s || !peak_running) return FMAP_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *peak_running = s->peak_running;
  return FMAP_OK;
}

fmap_status fmap_server_stats(fmap_server_t* s, int64_t* queued, int64_t* running,
                              int64_t* completed) {
  if (!s) return FMAP_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t run = 0;
  for (auto* r : s->slots) run += r != nullptr;
  if (queued) *queued = (int64_t)s->queue.size();
  if (running) *running = run;
  if (completed) *completed = s->completed;
  return FMAP_OK;
}

}  // extern "C"
