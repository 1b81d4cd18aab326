// Serving loop for the PEOs search: continuous batching with admission by device memory.
//
// Graph, codes and base stay resident.  Requests (a query, its k and efs) enter a host
// queue; a scheduler thread forms batches from the queue head and launches each with
// peos_search_batch on one of S streams, so up to S batches are on the GPU at once and
// requests that arrive while others run are admitted as soon as a stream and device
// memory are free.  Every batch takes one contiguous range of a device arena (its
// queries, per-query k and efs, results and search workspace); a batch is admitted only
// when the arena has room for it (first fit; ranges return to the arena when the batch's
// results are back on the host).  A load generator thread can replay timed arrivals.
// Each request's result depends only on the request (the search of a query never reads
// another query's state), so a request gets the same result alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

namespace peos {
namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size): free ranges sorted by offset, merged on release.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) { free_.push_back({0, size}); }
  bool alloc(size_t bytes, size_t* off) {
    bytes = up(bytes);
    for (size_t i = 0; i < free_.size(); ++i) {
      if (free_[i].len >= bytes) {
        *off = free_[i].off;
        free_[i].off += bytes;
        free_[i].len -= bytes;
        if (free_[i].len == 0) free_.erase(free_.begin() + i);
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = up(bytes);
    used_ -= bytes;
    auto it = std::lower_bound(free_.begin(), free_.end(), off,
                               [](const Range& r, size_t o) { return r.off < o; });
    it = free_.insert(it, {off, bytes});
    // merge with the next and the previous range
    if (it + 1 != free_.end() && it->off + it->len == (it + 1)->off) {
      it->len += (it + 1)->len;
      free_.erase(it + 1);
    }
    if (it != free_.begin() && (it - 1)->off + (it - 1)->len == it->off) {
      (it - 1)->len += it->len;
      free_.erase(it);
    }
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t size() const { return size_; }

 private:
  struct Range {
    size_t off, len;
  };
  size_t size_;
  size_t used_ = 0, peak_ = 0;
  std::vector<Range> free_;
};

struct Request {
  uint64_t id;
  int32_t k, ef;
  int64_t arrival_ns;
  std::vector<float> q;
};

struct Done {
  uint64_t id;
  int32_t k, status;
  int64_t arrival_ns, admit_ns, complete_ns;
  std::vector<int32_t> ids;
  std::vector<float> dists;
};

// One stream and its pinned host staging for batches of up to max_batch requests.
struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float* h_q = nullptr;
  int32_t* h_k = nullptr;
  int32_t* h_ef = nullptr;
  int32_t* h_ids = nullptr;
  float* h_d = nullptr;
  bool busy = false;
  size_t off = 0, bytes = 0;
  int64_t admit_ns = 0;
  std::vector<Request> reqs;
};

}  // namespace
}  // namespace peos

struct peos_server_s {
  int device = 0;
  peos_graph graph;
  peos_codes_t codes = nullptr;
  peos_matrix base, rerank;
  bool has_rerank = false;
  peos_server_config cfg;
  int d = 0;
  unsigned char* arena_mem = nullptr;
  peos::Arena* arena = nullptr;
  std::vector<peos::Slot> slots;

  std::mutex mu;
  std::condition_variable cv;
  std::deque<peos::Request> pending;
  std::deque<peos::Done> done;
  std::atomic<bool> stop{false};
  std::thread scheduler;
  std::thread generator;
  std::atomic<int64_t> gen_left{0};
  int64_t t0 = 0;
  // statistics
  uint64_t submitted = 0, completed = 0, batches = 0, batched_queries = 0, admission_waits = 0;
  int64_t failed = 0;
  peos_status last_launch_error = PEOS_OK;
};

namespace peos {
namespace {

// Device bytes of a batch of n requests: queries, k and efs, results, workspace.
size_t batch_bytes(peos_server_s* s, int64_t n, size_t* ws_out) {
  size_t ws = 0;
  peos_search_params p = s->cfg.params;
  p.k = s->cfg.k_max;
  p.ef = s->cfg.ef_max;
  if (peos_search_batch_workspace_size(&s->graph, s->codes, &s->base, s->has_rerank ? &s->rerank : nullptr, n, &p,
                                       &ws) != PEOS_OK)
    return (size_t)-1;
  if (ws_out) *ws_out = ws;
  return up((size_t)n * s->d * 4) + 2 * up((size_t)n * 4) + 2 * up((size_t)n * s->cfg.k_max * 4) + up(ws);
}

void finish_slot(peos_server_s* s, Slot& sl, peos_status st) {
  const int64_t t = now_ns() - s->t0;
  const int km = s->cfg.k_max;
  for (size_t i = 0; i < sl.reqs.size(); ++i) {
    Done r;
    r.id = sl.reqs[i].id;
    r.k = sl.reqs[i].k;
    r.status = st;
    r.arrival_ns = sl.reqs[i].arrival_ns;
    r.admit_ns = sl.admit_ns;
    r.complete_ns = t;
    r.ids.assign(sl.h_ids + i * km, sl.h_ids + (i + 1) * km);
    r.dists.assign(sl.h_d + i * km, sl.h_d + (i + 1) * km);
    s->done.push_back(std::move(r));
  }
  s->completed += sl.reqs.size();
  if (st != PEOS_OK) s->failed += (int64_t)sl.reqs.size();
  s->arena->release(sl.off, sl.bytes);
  sl.reqs.clear();
  sl.busy = false;
}

// Launch one batch on slot sl (called with the lock held; the requests are already
// moved into sl.reqs and their arena range reserved).
peos_status launch_slot(peos_server_s* s, Slot& sl, size_t ws) {
  const int64_t n = (int64_t)sl.reqs.size();
  const int d = s->d, km = s->cfg.k_max;
  for (int64_t i = 0; i < n; ++i) {
    std::memcpy(sl.h_q + i * d, sl.reqs[i].q.data(), sizeof(float) * d);
    sl.h_k[i] = sl.reqs[i].k;
    sl.h_ef[i] = sl.reqs[i].ef;
  }
  unsigned char* b = s->arena_mem + sl.off;
  float* dq = reinterpret_cast<float*>(b);
  size_t o = up((size_t)n * d * 4);
  int32_t* dk = reinterpret_cast<int32_t*>(b + o);
  o += up((size_t)n * 4);
  int32_t* def = reinterpret_cast<int32_t*>(b + o);
  o += up((size_t)n * 4);
  int32_t* dids = reinterpret_cast<int32_t*>(b + o);
  o += up((size_t)n * km * 4);
  float* dd = reinterpret_cast<float*>(b + o);
  o += up((size_t)n * km * 4);
  void* dws = b + o;
  cudaStream_t st = sl.stream;
  cudaError_t e = cudaMemcpyAsync(dq, sl.h_q, sizeof(float) * n * d, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dk, sl.h_k, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(def, sl.h_ef, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "server copy-in");
  peos_matrix Q{dq, nullptr, n, d, PEOS_F32};
  peos_search_params p = s->cfg.params;
  p.k = km;
  p.ef = s->cfg.ef_max;
  peos_status r = peos_search_batch(&s->graph, s->codes, &s->base, s->has_rerank ? &s->rerank : nullptr, &Q, &p, dk,
                                    def, dids, dd, nullptr, dws, ws, st);
  if (r != PEOS_OK) return r;
  e = cudaMemcpyAsync(sl.h_ids, dids, sizeof(int32_t) * n * km, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_d, dd, sizeof(float) * n * km, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
  if (e != cudaSuccess) return cuda_error(e, "server copy-out");
  return PEOS_OK;
}

void scheduler_main(peos_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (!s->stop.load()) {
    bool progress = false;
    // results of finished batches
    for (Slot& sl : s->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaSuccess) {
        finish_slot(s, sl, PEOS_OK);
        progress = true;
      } else if (q != cudaErrorNotReady) {  // the batch failed on the device
        s->last_launch_error = cuda_error(q, "server batch");
        finish_slot(s, sl, PEOS_E_CUDA);
        progress = true;
      }
    }
    // admit the queue head into free slots while the arena has room
    for (Slot& sl : s->slots) {
      if (sl.busy || s->pending.empty()) continue;
      int64_t n = std::min<int64_t>((int64_t)s->pending.size(), s->cfg.max_batch);
      size_t ws = 0, bytes = 0, off = 0;
      while (n > 0) {
        bytes = batch_bytes(s, n, &ws);
        if (bytes != (size_t)-1 && s->arena->alloc(bytes, &off)) break;
        n /= 2;
      }
      if (n == 0) {
        ++s->admission_waits;  // wait for memory to come back
        break;
      }
      sl.reqs.clear();
      for (int64_t i = 0; i < n; ++i) {
        sl.reqs.push_back(std::move(s->pending.front()));
        s->pending.pop_front();
      }
      sl.busy = true;
      sl.off = off;
      sl.bytes = bytes;
      sl.admit_ns = now_ns() - s->t0;
      ++s->batches;
      s->batched_queries += (uint64_t)n;
      peos_status st = launch_slot(s, sl, ws);
      if (st != PEOS_OK) {
        s->last_launch_error = st;
        cudaStreamSynchronize(sl.stream);
        finish_slot(s, sl, st);
      }
      progress = true;
    }
    if (progress) {
      s->cv.notify_all();
      continue;
    }
    bool inflight = false;
    for (Slot& sl : s->slots) inflight = inflight || sl.busy;
    // poll in-flight batches every few microseconds; sleep when idle
    s->cv.wait_for(lock, std::chrono::microseconds(inflight ? 5 : 200));
  }
  // drain: wait for every launched batch before the buffers go away
  for (Slot& sl : s->slots) {
    if (sl.busy) {
      cudaEventSynchronize(sl.done);
      finish_slot(s, sl, PEOS_OK);
    }
  }
}

bool valid_request(const peos_server_s* s, int32_t k, int32_t ef) {
  return k >= 1 && k <= s->cfg.k_max && ef >= k && ef <= s->cfg.ef_max;
}

peos_status push_request(peos_server_s* s, uint64_t id, const float* q, int32_t k, int32_t ef, int64_t arrival) {
  Request r;
  r.id = id;
  r.k = k;
  r.ef = ef;
  r.arrival_ns = arrival;
  r.q.assign(q, q + s->d);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->pending.push_back(std::move(r));
    ++s->submitted;
  }
  s->cv.notify_all();
  return PEOS_OK;
}

void destroy(peos_server_s* s) {
  if (s->generator.joinable()) {
    s->gen_left = 0;
    s->generator.join();
  }
  if (s->scheduler.joinable()) {
    s->stop = true;
    s->cv.notify_all();
    s->scheduler.join();
  }
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(s->device);
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    cudaFreeHost(sl.h_q);
    cudaFreeHost(sl.h_k);
    cudaFreeHost(sl.h_ef);
    cudaFreeHost(sl.h_ids);
    cudaFreeHost(sl.h_d);
  }
  cudaFree(s->arena_mem);
  delete s->arena;
  cudaSetDevice(cur);
  delete s;
}

}  // namespace
}  // namespace peos

using namespace peos;

extern "C" {

peos_status peos_server_create(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                               const peos_matrix* rerank, int32_t d, const peos_server_config* cfg,
                               peos_server_t* out) {
  if (!out || !cfg || !graph || !base) return set_error(PEOS_E_INVAL, "NULL argument");
  *out = nullptr;
  if (cfg->max_batch < 1 || cfg->streams < 1 || cfg->streams > 16)
    return set_error(PEOS_E_INVAL, "need max_batch >= 1 and 1 <= streams <= 16");
  if (cfg->k_max < 1 || cfg->ef_max < cfg->k_max) return set_error(PEOS_E_INVAL, "need 1 <= k_max <= ef_max");
  if (cfg->params.entries) return set_error(PEOS_E_INVAL, "the server takes no per-query entries");
  if (d != base->d) return set_error(PEOS_E_INVAL, "d != base.d");
  peos_server_s* s = new (std::nothrow) peos_server_s();
  if (!s) return set_error(PEOS_E_NOMEM, "host allocation");
  cudaGetDevice(&s->device);
  s->graph = *graph;
  s->codes = codes;
  s->base = *base;
  s->has_rerank = rerank != nullptr;
  if (rerank) s->rerank = *rerank;
  s->cfg = *cfg;
  s->d = d;
  // the largest batch must fit the arena, or nothing could ever be admitted
  const size_t one = batch_bytes(s, 1, nullptr);
  if (one == (size_t)-1) {
    std::string msg = peos_last_error();
    delete s;
    return set_error(PEOS_E_INVAL, "server: " + msg);
  }
  if (cfg->memory_budget < one) {
    delete s;
    return set_error(PEOS_E_INVAL, "memory_budget below the bytes of one request");
  }
  cudaError_t e = cudaMalloc(&s->arena_mem, cfg->memory_budget);
  if (e != cudaSuccess) {
    delete s;
    return cuda_error(e, "cudaMalloc(server arena)");
  }
  s->arena = new Arena(cfg->memory_budget);
  s->slots.resize(cfg->streams);
  const size_t mb = (size_t)cfg->max_batch;
  for (Slot& sl : s->slots) {
    e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_q, sizeof(float) * mb * d);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_k, sizeof(int32_t) * mb);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_ef, sizeof(int32_t) * mb);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_ids, sizeof(int32_t) * mb * cfg->k_max);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_d, sizeof(float) * mb * cfg->k_max);
    if (e != cudaSuccess) {
      destroy(s);
      return cuda_error(e, "server set-up");
    }
  }
  s->t0 = now_ns();
  s->scheduler = std::thread(scheduler_main, s);
  *out = s;
  return PEOS_OK;
}

peos_status peos_server_submit(peos_server_t s, uint64_t request_id, const float* query, int32_t k, int32_t ef) {
  if (!s || !query) return set_error(PEOS_E_INVAL, "NULL argument");
  if (!valid_request(s, k, ef)) return set_error(PEOS_E_INVAL, "need 1 <= k <= ef, k <= k_max, ef <= ef_max");
  return push_request(s, request_id, query, k, ef, now_ns() - s->t0);
}

peos_status peos_server_replay(peos_server_t s, int64_t n, const uint64_t* request_ids, const float* queries,
                               const int32_t* k, const int32_t* ef, const int64_t* arrival_ns) {
  if (!s || (n > 0 && (!request_ids || !queries || !k || !ef || !arrival_ns)))
    return set_error(PEOS_E_INVAL, "NULL argument");
  for (int64_t i = 0; i < n; ++i) {
    if (!valid_request(s, k[i], ef[i]))
      return set_error(PEOS_E_INVAL, "request " + std::to_string(i) + ": need 1 <= k <= ef, k <= k_max, ef <= ef_max");
    if (i > 0 && arrival_ns[i] < arrival_ns[i - 1]) return set_error(PEOS_E_INVAL, "arrival times must ascend");
  }
  if (s->generator.joinable()) {
    if (s->gen_left.load() > 0) return set_error(PEOS_E_INVAL, "a replay is still running");
    s->generator.join();
  }
  std::vector<uint64_t> ids(request_ids, request_ids + n);
  std::vector<float> qs(queries, queries + (size_t)n * s->d);
  std::vector<int32_t> ks(k, k + n), efs(ef, ef + n);
  std::vector<int64_t> at(arrival_ns, arrival_ns + n);
  s->gen_left = n;
  s->generator = std::thread([s, ids = std::move(ids), qs = std::move(qs), ks = std::move(ks),
                              efs = std::move(efs), at = std::move(at)]() {
    const int64_t start = now_ns();
    for (size_t i = 0; i < ids.size() && s->gen_left.load() > 0; ++i) {
      const int64_t due = start + at[i];
      // sleep until shortly before the arrival, then spin for the last microseconds
      for (;;) {
        const int64_t left = due - now_ns();
        if (left <= 0) break;
        if (left > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(left - 100000));
        else std::this_thread::yield();
      }
      push_request(s, ids[i], qs.data() + i * s->d, ks[i], efs[i], due - s->t0);
      --s->gen_left;
    }
    s->gen_left = 0;
  });
  return PEOS_OK;
}

peos_status peos_server_poll(peos_server_t s, int32_t max_results, peos_server_result* results, int32_t* ids_out,
                             float* dists_out, int32_t* n_out, int32_t wait_us) {
  if (!s || !n_out || (max_results > 0 && (!results || !ids_out || !dists_out)))
    return set_error(PEOS_E_INVAL, "NULL argument");
  std::unique_lock<std::mutex> lock(s->mu);
  if (s->done.empty() && wait_us > 0)
    s->cv.wait_for(lock, std::chrono::microseconds(wait_us), [s] { return !s->done.empty(); });
  int32_t n = 0;
  const int km = s->cfg.k_max;
  while (n < max_results && !s->done.empty()) {
    Done& r = s->done.front();
    results[n] = peos_server_result{r.id, r.k, r.status, r.arrival_ns, r.admit_ns, r.complete_ns};
    std::memcpy(ids_out + (size_t)n * km, r.ids.data(), sizeof(int32_t) * km);
    std::memcpy(dists_out + (size_t)n * km, r.dists.data(), sizeof(float) * km);
    s->done.pop_front();
    ++n;
  }
  *n_out = n;
  return PEOS_OK;
}

peos_status peos_server_stats(peos_server_t s, peos_server_stats_t* out) {
  if (!s || !out) return set_error(PEOS_E_INVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = (uint64_t)s->failed;
  out->pending = s->pending.size();
  out->batches = s->batches;
  out->batched_queries = s->batched_queries;
  out->admission_waits = s->admission_waits;
  out->arena_bytes = s->arena->size();
  out->arena_used = s->arena->used();
  out->arena_peak = s->arena->peak();
  int busy = 0;
  for (const Slot& sl : s->slots) busy += sl.busy ? 1 : 0;
  out->batches_in_flight = busy;
  out->last_error = s->last_launch_error;
  return PEOS_OK;
}

peos_status peos_server_destroy(peos_server_t s) {
  if (!s) return PEOS_OK;
  destroy(s);
  return PEOS_OK;
}

}  // extern "C"
