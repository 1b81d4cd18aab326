// C ABI of the PEOs library (declared in include/peos.h): argument validation,
// ownership of the index data, stream-ordered scratch, and the host-side
// constants of the routing test.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace peos {

namespace {
thread_local std::string g_last_error;

bool valid_dtype_f32(const peos_matrix* M) { return M->dtype == PEOS_F32; }

}  // namespace

peos_status set_error(peos_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

peos_status cuda_error(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return set_error(PEOS_E_CUDA, m);
}

// Phi^{-1}(p) by bisection of Phi(x) = erfc(-x / sqrt 2) / 2 down to adjacent doubles.
double norm_ppf(double p) {
  double lo = -40.0, hi = 40.0;
  while (true) {
    const double mid = lo + 0.5 * (hi - lo);
    if (mid <= lo || mid >= hi) break;
    const double cdf = 0.5 * erfc(-mid * 0.7071067811865476);
    if (cdf < p) lo = mid; else hi = mid;
  }
  return lo + 0.5 * (hi - lo);
}

// mode 0: sqrt(2 ln m); mode 1: E[max_j |g_j|] over m iid N(0,1) = int_0^inf (1 - erf(x/sqrt2)^m) dx,
// trapezoid rule on [0, 40] with step 1e-4 (the integrand is smooth and decays like a Gaussian tail).
// The quadrature is computed once per m and cached.
double eta_value(int m, int mode) {
  if (mode == 0) return sqrt(2.0 * log((double)m));
  static std::mutex mu;
  static double cache[128] = {0};
  std::lock_guard<std::mutex> lock(mu);
  if (m >= 2 && m < 128 && cache[m] > 0) return cache[m];
  const double h = 1e-4;
  const int steps = 400000;
  double s = 0.5 * (1.0 - pow(erf(0.0), (double)m));
  for (int i = 1; i < steps; ++i) s += 1.0 - pow(erf(i * h * 0.7071067811865476), (double)m);
  s += 0.5 * (1.0 - pow(erf(steps * h * 0.7071067811865476), (double)m));
  s *= h;
  if (m >= 2 && m < 128) cache[m] = s;
  return s;
}

}  // namespace peos

using namespace peos;

namespace peos_api_detail {

peos_status check_graph(const peos_graph* g) {
  if (!g) return set_error(PEOS_E_INVAL, "graph is NULL");
  if (!g->nbrs && g->n > 0) return set_error(PEOS_E_INVAL, "graph.nbrs is NULL");
  if (g->n < 1) return set_error(PEOS_E_INVAL, "graph.n must be >= 1");
  if (g->n > 0x7fffffffLL) return set_error(PEOS_E_INVAL, "graph.n must fit int32 ids");
  if (g->R < 1 || g->R > kMaxR) return set_error(PEOS_E_INVAL, "graph.R must be in 1..64");
  if (g->entry < 0 || (int64_t)g->entry >= g->n) return set_error(PEOS_E_INVAL, "graph.entry outside [0, n)");
  return PEOS_OK;
}

// `stored` = the matrix may hold reduced-precision rows (the base a search reads);
// everything else is FP32.
peos_status check_matrix(const peos_matrix* M, const char* name, bool stored = false) {
  if (!M) return set_error(PEOS_E_INVAL, std::string(name) + " is NULL");
  if (M->n < 0 || M->d < 1) return set_error(PEOS_E_INVAL, std::string(name) + ": bad shape");
  if (M->n > 0 && !M->data) return set_error(PEOS_E_INVAL, std::string(name) + ".data is NULL");
  if (M->dtype != PEOS_F32 && M->dtype != PEOS_BF16 && M->dtype != PEOS_FP8E4M3)
    return set_error(PEOS_E_INVAL, std::string(name) + ": unknown dtype");
  if (!stored && !valid_dtype_f32(M)) return set_error(PEOS_E_INVAL, std::string(name) + ": must be PEOS_F32");
  if (M->dtype == PEOS_FP8E4M3 && M->n > 0 && !M->scales)
    return set_error(PEOS_E_INVAL, std::string(name) + ": PEOS_FP8E4M3 rows need per-row scales");
  if (M->dtype != PEOS_FP8E4M3 && M->scales)
    return set_error(PEOS_E_INVAL, std::string(name) + ": scales are only used with PEOS_FP8E4M3");
  if (M->scales && ((uintptr_t)M->scales & 3) != 0)
    return set_error(PEOS_E_INVAL, std::string(name) + ".scales not 4-byte aligned");
  if (M->d % 4 != 0) return set_error(PEOS_E_UNSUPPORTED, std::string(name) + ": d must be a multiple of 4");
  if (((uintptr_t)M->data & 15) != 0) return set_error(PEOS_E_INVAL, std::string(name) + ".data not 16-byte aligned");
  return PEOS_OK;
}

__global__ void count_bad_ids(const int32_t* nbrs, long long total, long long n, unsigned long long* bad) {
  unsigned long long local = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int32_t u = nbrs[i];
    if (u < -1 || (long long)u >= n) ++local;
  }
  if (local) atomicAdd(bad, local);
}

int auto_hash_bits(int ef) {
  int want = 16 * ef;
  if (want < 512) want = 512;
  if (want > 4096) want = 4096;
  int b = 0;
  while ((1 << b) < want) ++b;
  return b;
}

// Per-call scratch comes from the device's default memory pool.  The pool is told
// once per device to keep freed memory (release threshold = max) so that repeated
// searches reuse it instead of mapping it again on every call.
void keep_pool_memory() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t threshold = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
  }
  done[dev] = true;
}

struct StreamScratch {
  void* p = nullptr;
  cudaStream_t st;
  explicit StreamScratch(cudaStream_t s) : st(s) {}
  cudaError_t alloc(size_t bytes) {
    keep_pool_memory();
    return cudaMallocAsync(&p, bytes, st);
  }
  ~StreamScratch() {
    if (p) cudaFreeAsync(p, st);
  }
};

// Stage tracing: a pool of events, the calls recorded since the last read, and the
// running totals.
struct Tracer {
  std::mutex mu;
  bool on = false;
  std::vector<std::pair<int, cudaEvent_t>> pool;  // (device, event)
  std::vector<peos::TraceCall> pending;
};
Tracer& tracer() {
  static Tracer t;
  return t;
}

}  // namespace peos_api_detail

using namespace peos_api_detail;

bool peos::trace_begin(TraceCall* tc) {
  Tracer& t = tracer();
  std::lock_guard<std::mutex> lock(t.mu);
  if (!t.on) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  tc->device = dev;
  for (int i = 0; i <= PEOS_NSTAGES; ++i) {
    cudaEvent_t e = nullptr;
    for (size_t j = 0; j < t.pool.size(); ++j) {
      if (t.pool[j].first == dev) {
        e = t.pool[j].second;
        t.pool.erase(t.pool.begin() + j);
        break;
      }
    }
    if (!e && cudaEventCreate(&e) != cudaSuccess) {
      for (int k = 0; k < i; ++k) t.pool.push_back({dev, tc->ev[k]});
      return false;
    }
    tc->ev[i] = e;
  }
  return true;
}

void peos::trace_end(const TraceCall& tc) {
  Tracer& t = tracer();
  std::lock_guard<std::mutex> lock(t.mu);
  t.pending.push_back(tc);
}

namespace peos_api_detail {

// Workspace of a batch call: [work counter | query tables | re-rank lists (ids, dists) | order].
struct BatchLayout {
  size_t tables, rr_ids, rr_dists, order, total;
};
BatchLayout batch_layout(const SearchLaunch& a, int64_t nq, bool rerank) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  BatchLayout L;
  L.tables = 256;
  L.rr_ids = L.tables + up(search_scratch_bytes(nq, a.L, a.m, a.routing));
  const size_t lb = rerank ? (size_t)nq * a.ef * sizeof(int32_t) : 0;
  L.rr_dists = L.rr_ids + up(lb);
  L.order = L.rr_dists + up(lb);
  L.total = L.order + up((size_t)nq * sizeof(int32_t));
  return L;
}

peos_status check_rerank(const peos_matrix* rerank, const peos_matrix* base, const SearchLaunch& a) {
  if (!rerank) return PEOS_OK;
  peos_status st = check_matrix(rerank, "rerank");
  if (st) return st;
  if (rerank->n != base->n || rerank->d != base->d) return set_error(PEOS_E_INVAL, "rerank shape != base shape");
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (search_rerank_smem(a.d, a.ef) > (size_t)maxsm)
    return set_error(PEOS_E_UNSUPPORTED, "re-rank shared memory exceeds the per-CTA limit (lower ef)");
  return PEOS_OK;
}

}  // namespace peos_api_detail

peos_status peos::check_matrix_public(const peos_matrix* M, const char* name) { return check_matrix(M, name); }

extern "C" {

const char* peos_last_error(void) { return g_last_error.c_str(); }

peos_status peos_trace_enable(int32_t on) {
  Tracer& t = tracer();
  std::lock_guard<std::mutex> lock(t.mu);
  t.on = on != 0;
  return PEOS_OK;
}

peos_status peos_trace_read(double* ms, int64_t* calls) {
  if (!ms || !calls) return set_error(PEOS_E_INVAL, "NULL output");
  Tracer& t = tracer();
  std::vector<TraceCall> done;
  {
    std::lock_guard<std::mutex> lock(t.mu);
    done.swap(t.pending);
  }
  for (int i = 0; i < PEOS_NSTAGES; ++i) ms[i] = 0.0;
  *calls = 0;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaError_t first = cudaSuccess;
  for (const TraceCall& c : done) {
    cudaSetDevice(c.device);
    cudaError_t e = cudaEventSynchronize(c.ev[PEOS_NSTAGES]);
    for (int i = 0; e == cudaSuccess && i < PEOS_NSTAGES; ++i) {
      float x = 0.0f;
      e = cudaEventElapsedTime(&x, c.ev[i], c.ev[i + 1]);
      ms[i] += x;
    }
    if (e == cudaSuccess) ++*calls;
    else if (first == cudaSuccess) first = e;
  }
  cudaSetDevice(cur);
  {
    std::lock_guard<std::mutex> lock(t.mu);
    for (const TraceCall& c : done)
      for (int i = 0; i <= PEOS_NSTAGES; ++i) t.pool.push_back({c.device, c.ev[i]});
  }
  if (first != cudaSuccess) return cuda_error(first, "peos_trace_read");
  return PEOS_OK;
}

const char* peos_version(void) {
#ifdef PEOS_CHECKED
  return "peos-gb300 0.1 (sm_103a, self-checked)";
#else
  return "peos-gb300 0.1 (sm_103a)";
#endif
}

peos_status peos_check_read(uint64_t* counts) {
  if (!counts) return set_error(PEOS_E_INVAL, "NULL argument");
#ifdef PEOS_CHECKED
  unsigned long long* c = check_counters();
  if (!c) return set_error(PEOS_E_NOMEM, "violation counters");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(counts, c, PEOS_CHECK_KINDS * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(c, 0, PEOS_CHECK_KINDS * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_error(e, "peos_check_read");
  return PEOS_OK;
#else
  for (int i = 0; i < PEOS_CHECK_KINDS; ++i) counts[i] = 0;
  return set_error(PEOS_E_UNSUPPORTED, "this library was built without PEOS_CHECKED");
#endif
}

peos_status peos_projections(uint64_t seed, int32_t d, int32_t L, int32_t m, float* A_host, float* B_host) {
  if (!A_host || !B_host) return set_error(PEOS_E_INVAL, "NULL output");
  if (d < 1 || L < 1 || d % L != 0) return set_error(PEOS_E_INVAL, "need d >= 1, L >= 1, d % L == 0");
  if (m < 2 || m > 127) return set_error(PEOS_E_INVAL, "m must be in 2..127");
  projections_host(seed, d, L, m, A_host, B_host);
  return PEOS_OK;
}

peos_status peos_build_codes(const peos_graph* graph, const peos_matrix* base, int32_t L, int32_t m, uint64_t seed,
                             void* stream, peos_codes_t* out) {
  return peos_build_codes_permuted(graph, base, L, m, seed, nullptr, stream, out);
}

peos_status peos_build_codes_compact(const peos_graph* graph, const peos_matrix* base, int32_t L, int32_t m,
                                     uint64_t seed, int32_t scalar_bits, void* stream, peos_codes_t* out) {
  NvtxRange nvtx_range("peos.build_codes");
  if (!out) return set_error(PEOS_E_INVAL, "out is NULL");
  *out = nullptr;
  if (scalar_bits != 32 && scalar_bits != 16 && scalar_bits != 8)
    return set_error(PEOS_E_INVAL, "scalar_bits must be 32, 16 or 8");
  peos_codes_t c = nullptr;
  peos_status st = peos_build_codes_permuted(graph, base, L, m, seed, nullptr, stream, &c);
  if (st) return st;
  if (scalar_bits == 32) {
    *out = c;
    return PEOS_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t stride = record_stride(c->R, c->L, c->m, scalar_bits);
  uint8_t* rec = nullptr;
  if (cudaMalloc(&rec, (size_t)(c->n > 0 ? c->n : 1) * stride) != cudaSuccess) {
    peos_codes_free(c);
    return set_error(PEOS_E_NOMEM, "cudaMalloc compact records");
  }
  cudaError_t e = launch_compact_records(c->records, c->rec_stride, c->n, c->R, code_words(c->L, c->m), c->node_proj,
                                         table_stride(c->L, c->m), c->L, c->m, scalar_bits, rec, stride, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(rec);
    peos_codes_free(c);
    return cuda_error(e, "peos_build_codes_compact");
  }
  cudaFree(c->records);
  c->records = rec;
  c->rec_stride = stride;
  c->scalar_bits = scalar_bits;
  *out = c;
  return PEOS_OK;
}

peos_status peos_dim_permutation(const peos_graph* graph, const peos_matrix* base, int32_t L, int32_t* perm,
                                 void* stream) {
  NvtxRange nvtx_range("peos.dim_permutation");
  peos_status st = check_graph(graph);
  if (st) return st;
  st = check_matrix(base, "base");
  if (st) return st;
  if (base->n != graph->n) return set_error(PEOS_E_INVAL, "base.n != graph.n");
  if (!perm) return set_error(PEOS_E_INVAL, "perm is NULL");
  const int d = base->d;
  if (L < 1 || d % L != 0) return set_error(PEOS_E_INVAL, "L must divide d (space partition, Sec. 4.1)");
  if (d > 2048) return set_error(PEOS_E_UNSUPPORTED, "the permutation supports d <= 2048");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, dim_perm_scratch_bytes(d), s);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync");
  e = launch_dim_permutation(static_cast<const float*>(base->data), graph->n, d, graph->nbrs, graph->R, L, scratch,
                             perm, s);
  cudaError_t f = cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = f;
  if (e != cudaSuccess) return cuda_error(e, "peos_dim_permutation");
  return PEOS_OK;
}

peos_status peos_build_codes_permuted(const peos_graph* graph, const peos_matrix* base, int32_t L, int32_t m,
                                      uint64_t seed, const int32_t* perm, void* stream, peos_codes_t* out) {
  NvtxRange nvtx_range("peos.build_codes");
  if (!out) return set_error(PEOS_E_INVAL, "out is NULL");
  *out = nullptr;
  peos_status st = check_graph(graph);
  if (st) return st;
  st = check_matrix(base, "base");
  if (st) return st;
  if (base->n != graph->n) return set_error(PEOS_E_INVAL, "base.n != graph.n");
  const int d = base->d;
  if (L < 1 || d % L != 0) return set_error(PEOS_E_INVAL, "L must divide d (space partition, Sec. 4.1)");
  if (m < 2 || m > 127) return set_error(PEOS_E_INVAL, "m must be in 2..127 (signed 8-bit codes)");
  if (code_words(L, m) > kMaxCodeWords)
    return set_error(PEOS_E_UNSUPPORTED, "too many codes per edge: need (L + 1) <= 3 * codes_per_word(m)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = graph->n;
  const int R = graph->R;

  // reject out-of-range ids before anything reads through them
  {
    unsigned long long* bad = nullptr;
    cudaError_t e = cudaMallocAsync(&bad, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync");
    cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
    count_bad_ids<<<256, 256, 0, s>>>(graph->nbrs, n * R, n, bad);
    unsigned long long h = 0;
    cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(bad, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "graph validation");
    if (h) return set_error(PEOS_E_INVAL, "graph.nbrs holds ids outside [-1, n)");
  }

  peos_codes_s* c = new (std::nothrow) peos_codes_s();
  if (!c) return set_error(PEOS_E_NOMEM, "host allocation");
  cudaGetDevice(&c->device);
  c->n = n;
  c->R = R;
  c->L = L;
  c->m = m;
  c->d = d;
  c->entry = graph->entry;
  c->seed = seed;
  c->rec_stride = record_stride(R, L, m);
  const int dp = d / L;
  std::vector<float> hA((size_t)L * m * dp), hB((size_t)m * d);
  projections_host(seed, d, L, m, hA.data(), hB.data());
  // k-major copy: the lanes that build the entries j of one block read consecutive floats
  std::vector<float> hW((size_t)2 * d * m);
  for (int j = 0; j < m; ++j)
    for (int k = 0; k < d; ++k) hW[(size_t)k * m + j] = hB[(size_t)j * d + k];
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < m; ++j)
      for (int k = 0; k < dp; ++k)
        hW[(size_t)d * m + ((size_t)i * dp + k) * m + j] = hA[((size_t)i * m + j) * dp + k];
  auto fail = [&](peos_status code, const std::string& msg) {
    cudaFree(c->records);
    cudaFree(c->node_proj);
    cudaFree(c->A);
    cudaFree(c->B);
    cudaFree(c->Wt);
    cudaFree(c->perm);
    cudaFree(c->norms);
    delete c;
    return set_error(code, msg);
  };
  cudaError_t e;
  if (perm) {
    // the permutation must be one: every coordinate exactly once
    std::vector<int32_t> hp(d);
    e = cudaMemcpyAsync(hp.data(), perm, (size_t)d * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_error(e, "reading perm"), g_last_error);
    std::vector<char> seen(d, 0);
    for (int t = 0; t < d; ++t) {
      if (hp[t] < 0 || hp[t] >= d || seen[hp[t]]) return fail(PEOS_E_INVAL, "perm is not a permutation of 0..d-1");
      seen[hp[t]] = 1;
    }
    if ((e = cudaMalloc(&c->perm, (size_t)d * sizeof(int32_t))) != cudaSuccess)
      return fail(PEOS_E_NOMEM, "cudaMalloc perm");
    e = cudaMemcpyAsync(c->perm, hp.data(), (size_t)d * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(cuda_error(e, "copying perm"), g_last_error);
  }
  if ((e = cudaMalloc(&c->A, hA.size() * sizeof(float))) != cudaSuccess) return fail(PEOS_E_NOMEM, "cudaMalloc A");
  if ((e = cudaMalloc(&c->B, hB.size() * sizeof(float))) != cudaSuccess) return fail(PEOS_E_NOMEM, "cudaMalloc B");
  if ((e = cudaMalloc(&c->Wt, hW.size() * sizeof(float))) != cudaSuccess) return fail(PEOS_E_NOMEM, "cudaMalloc Wt");
  if ((e = cudaMalloc(&c->records, (size_t)n * c->rec_stride)) != cudaSuccess)
    return fail(PEOS_E_NOMEM, "cudaMalloc records");
  if ((e = cudaMalloc(&c->node_proj, (size_t)n * table_stride(L, m) * sizeof(float))) != cudaSuccess)
    return fail(PEOS_E_NOMEM, "cudaMalloc node_proj");
  if ((e = cudaMalloc(&c->norms, (size_t)(n > 0 ? n : 1) * sizeof(float))) != cudaSuccess)
    return fail(PEOS_E_NOMEM, "cudaMalloc norms");
  e = cudaMemcpyAsync(c->A, hA.data(), hA.size() * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->B, hB.data(), hB.size() * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->Wt, hW.data(), hW.size() * sizeof(float), cudaMemcpyHostToDevice, s);
  // node tables first: the code builder reads t(v) for each edge's node term
  if (e == cudaSuccess)
    e = launch_node_proj(static_cast<const float*>(base->data), n, d, L, m, c->A, c->B, c->perm, c->node_proj,
                         table_stride(L, m), s);
  if (e == cudaSuccess)
    e = launch_build_codes(static_cast<const float*>(base->data), n, d, graph->nbrs, R, L, m, c->A, c->B, c->perm,
                           c->node_proj, table_stride(L, m), c->records, c->rec_stride, s);
  if (e == cudaSuccess) e = launch_row_norms(static_cast<const float*>(base->data), n, d, c->norms, s);
  // the host vectors hA/hB go out of scope: wait for their copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    peos_status r = cuda_error(e, "peos_build_codes");
    std::string msg = g_last_error;
    return fail(r, msg);
  }
  if (peos_status r = attach_wide_flags(c, s)) {
    std::string msg = g_last_error;
    return fail(r, msg);
  }
  *out = c;
  return PEOS_OK;
}

peos_status peos_build_simhash(const peos_graph* graph, const peos_matrix* base, int32_t K, uint64_t seed,
                               void* stream, peos_codes_t* out) {
  NvtxRange nvtx_range("peos.build_simhash");
  if (!out) return set_error(PEOS_E_INVAL, "out is NULL");
  *out = nullptr;
  peos_status st = check_graph(graph);
  if (st) return st;
  st = check_matrix(base, "base");
  if (st) return st;
  if (base->n != graph->n) return set_error(PEOS_E_INVAL, "base.n != graph.n");
  if (K < 64 || K > kMaxSimHashBits || K % 64 != 0) return set_error(PEOS_E_INVAL, "K must be 64, 128 or 192");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = graph->n;
  const int R = graph->R, d = base->d;
  {
    unsigned long long* bad = nullptr;
    cudaError_t e = cudaMallocAsync(&bad, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync");
    cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
    count_bad_ids<<<256, 256, 0, s>>>(graph->nbrs, n * R, n, bad);
    unsigned long long h = 0;
    cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(bad, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "graph validation");
    if (h) return set_error(PEOS_E_INVAL, "graph.nbrs holds ids outside [-1, n)");
  }
  peos_codes_s* c = new (std::nothrow) peos_codes_s();
  if (!c) return set_error(PEOS_E_NOMEM, "host allocation");
  cudaGetDevice(&c->device);
  c->kind = kCodesSimHash;
  c->n = n;
  c->R = R;
  c->L = 1;
  c->m = K;
  c->d = d;
  c->entry = graph->entry;
  c->seed = seed;
  c->rec_stride = record_stride_words(R, K / 64);
  // the K vectors S_i ~ N(0, I_d): the b_j of the projection generator with L = 1, m = K
  std::vector<float> hA((size_t)K * d), hS((size_t)K * d);
  projections_host(seed, d, 1, K, hA.data(), hS.data());
  auto fail = [&](peos_status code, const std::string& msg) {
    cudaFree(c->records);
    cudaFree(c->node_proj);
    cudaFree(c->B);
    delete c;
    return set_error(code, msg);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&c->B, hS.size() * sizeof(float))) != cudaSuccess) return fail(PEOS_E_NOMEM, "cudaMalloc S");
  if ((e = cudaMalloc(&c->records, (size_t)n * c->rec_stride)) != cudaSuccess)
    return fail(PEOS_E_NOMEM, "cudaMalloc records");
  if ((e = cudaMalloc(&c->node_proj, (size_t)n * K * sizeof(float))) != cudaSuccess)
    return fail(PEOS_E_NOMEM, "cudaMalloc node table");
  e = cudaMemcpyAsync(c->B, hS.data(), hS.size() * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_simhash_build(static_cast<const float*>(base->data), n, d, graph->nbrs, R, K, c->B, c->records,
                             c->rec_stride, c->node_proj, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    peos_status r = cuda_error(e, "peos_build_simhash");
    std::string msg = g_last_error;
    return fail(r, msg);
  }
  if (peos_status r = attach_wide_flags(c, s)) {
    std::string msg = g_last_error;
    return fail(r, msg);
  }
  *out = c;
  return PEOS_OK;
}

peos_status peos_codes_free(peos_codes_t c) {
  if (!c) return PEOS_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  cudaFree(c->records);
  cudaFree(c->node_proj);
  cudaFree(c->A);
  cudaFree(c->B);
  cudaFree(c->Wt);
  cudaFree(c->perm);
  cudaFree(c->norms);
  cudaFree(c->wide);
  cudaSetDevice(cur);
  delete c;
  return PEOS_OK;
}

peos_status peos_codes_get_info(peos_codes_t c, peos_codes_info* info) {
  if (!c || !info) return set_error(PEOS_E_INVAL, "NULL argument");
  info->n = c->n;
  info->R = c->R;
  info->L = c->L;
  info->m = c->m;
  info->d = c->d;
  info->entry = c->entry;
  info->record_stride = c->rec_stride;
  info->records = c->records;
  info->node_proj = c->node_proj;
  info->node_proj_stride = node_table_stride(c);
  info->kind = c->kind;
  info->A = c->A;
  info->B = c->B;
  info->perm = c->perm;
  info->norms = c->norms;
  info->scalar_bits = c->kind == kCodesPeos ? c->scalar_bits : 32;
  return PEOS_OK;
}

peos_status peos_codes_export(peos_codes_t c, void* records_host, float* node_proj_host, float* A_host,
                              float* B_host) {
  if (!c) return set_error(PEOS_E_INVAL, "NULL codes");
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(c->device);
  cudaError_t e = cudaDeviceSynchronize();
  const size_t tw = (size_t)node_table_stride(c);
  if (e == cudaSuccess && records_host)
    e = cudaMemcpy(records_host, c->records, (size_t)c->n * c->rec_stride, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && node_proj_host)
    e = cudaMemcpy(node_proj_host, c->node_proj, (size_t)c->n * tw * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && A_host && c->A)
    e = cudaMemcpy(A_host, c->A, (size_t)c->m * c->d * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && B_host) e = cudaMemcpy(B_host, c->B, (size_t)c->m * c->d * sizeof(float), cudaMemcpyDeviceToHost);
  cudaSetDevice(cur);
  if (e != cudaSuccess) return cuda_error(e, "peos_codes_export");
  return PEOS_OK;
}

}  // extern "C"

peos_status peos::prepare_search(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base, int64_t nq,
                                 int d_q, const peos_search_params* P, SearchLaunch* a) {
  peos_status st = check_graph(graph);
  if (st) return st;
  st = check_matrix(base, "base", /*stored=*/true);
  if (st) return st;
  if (!P) return set_error(PEOS_E_INVAL, "params is NULL");
  if (base->n != graph->n) return set_error(PEOS_E_INVAL, "base.n != graph.n");
  if (d_q != base->d) return set_error(PEOS_E_INVAL, "queries.d != base.d");
  if (nq < 0) return set_error(PEOS_E_INVAL, "nq < 0");
  if (P->k < 1 || P->ef < P->k || P->ef > kMaxEf) return set_error(PEOS_E_INVAL, "need 1 <= k <= ef <= 1024");
  if (P->routing < 0 || P->routing > 2) return set_error(PEOS_E_INVAL, "routing must be 0, 1 or 2");
  if (P->test_mode < 0 || P->test_mode > 3) return set_error(PEOS_E_INVAL, "test_mode must be 0..3");
  if (P->test_mode == 3 && (P->routing != 1 || P->frame != 1))
    return set_error(PEOS_E_INVAL, "test_mode 3 (the quantile table) is a form of the frame-Q PEOs test");
  if (P->eta_mode != 0 && P->eta_mode != 1) return set_error(PEOS_E_INVAL, "eta_mode must be 0 or 1");
  if (P->frame != 0 && P->frame != 1) return set_error(PEOS_E_INVAL, "frame must be 0 or 1");
  if (P->frame == 1 && P->routing != 1) return set_error(PEOS_E_INVAL, "frame Q is a form of the PEOs test (routing 1)");
  if (P->frame == 1 && base->dtype != PEOS_F32) return set_error(PEOS_E_UNSUPPORTED, "frame Q reads FP32 rows only");
  int hb = 0, hb_min = 0;
  if (P->visited_slots == 0) {
    hb = auto_hash_bits(P->ef);
    hb_min = 9;  // the launcher may lower an automatic table to 512 slots (run_search)
  } else {
    const int vsl = P->visited_slots;
    if (vsl < 256 || vsl > 16384 || (vsl & (vsl - 1)))
      return set_error(PEOS_E_INVAL, "visited_slots must be a power of two in 256..16384");
    while ((1 << hb) < vsl) ++hb;
  }
  int warps = P->warps_per_cta == 0 ? 8 : P->warps_per_cta;
  if (warps < 1 || warps > 8) return set_error(PEOS_E_INVAL, "warps_per_cta must be in 1..8");
  if (P->gather_rows != 0 && P->gather_rows != 4 && P->gather_rows != 8)
    return set_error(PEOS_E_INVAL, "gather_rows must be 0, 4 or 8");
  const int beam = P->beam == 0 ? 1 : P->beam;
  if (beam != 1 && beam != 2 && beam != 4) return set_error(PEOS_E_INVAL, "beam must be 0, 1, 2 or 4");
  if (beam > 1 && (P->routing == 2 || (P->routing == 1 && (P->frame != 0 || (codes && codes->perm) ||
                                                           (codes && codes->scalar_bits != 32)))))
    return set_error(PEOS_E_UNSUPPORTED,
                     "beam 2 / 4 is built for plain routing and PEOs in frame T with FP32 scalars, unpermuted");
  *a = SearchLaunch{};
  a->gather = P->gather_rows;
  a->beam = beam;
  if (P->routing == 2) {
    if (!codes || codes->kind != kCodesSimHash) return set_error(PEOS_E_INVAL, "SimHash routing needs SimHash codes");
    if (!(P->eps > 0.0f && P->eps < 1.0f)) return set_error(PEOS_E_INVAL, "eps must be in (0, 1)");
    if (codes->n != graph->n || codes->R != graph->R || codes->d != base->d)
      return set_error(PEOS_E_INVAL, "codes were built for another graph/base shape");
    if (base->dtype != PEOS_F32) return set_error(PEOS_E_UNSUPPORTED, "SimHash routing reads FP32 rows only");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != codes->device) return set_error(PEOS_E_INVAL, "codes live on another device");
    a->rec = codes->records;
    a->rec_stride = codes->rec_stride;
    a->B = codes->B;
    a->L = 1;
    a->m = codes->m;
    a->sh_K = codes->m;
    a->sh_tv = codes->node_proj;
    simhash_acrit(codes->m, (double)P->eps, a->sh_acrit);
  }
  if (P->routing == 1) {
    if (!codes) return set_error(PEOS_E_INVAL, "PEOs routing needs codes");
    if (codes->kind != kCodesPeos) return set_error(PEOS_E_INVAL, "PEOs routing needs PEOs codes");
    if (!(P->eps > 0.0f && P->eps <= 0.5f)) return set_error(PEOS_E_INVAL, "eps must be in (0, 0.5] (Theorem 5.3)");
    if (codes->n != graph->n || codes->R != graph->R || codes->d != base->d)
      return set_error(PEOS_E_INVAL, "codes were built for another graph/base shape");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != codes->device) return set_error(PEOS_E_INVAL, "codes live on another device");
    if (codes->scalar_bits != 32 && (P->frame != 0 || codes->perm))
      return set_error(PEOS_E_UNSUPPORTED, "codes with 8/16-bit scalars are searched in frame T");
    a->scalar_bits = codes->scalar_bits;
    a->rec = codes->records;
    a->rec_stride = codes->rec_stride;
    a->tv_stride = table_stride(codes->L, codes->m);
    a->A = codes->A;
    a->B = codes->B;
    a->Wt = codes->Wt;
    a->perm = codes->perm;
    a->frame = P->frame;
    a->norms = codes->norms;
    a->L = codes->L;
    a->m = codes->m;
    a->z_eps = (float)norm_ppf((double)P->eps);
    a->c_eta = (float)(sqrt((double)codes->L) * eta_value(codes->m, P->eta_mode));
  }
  a->X = base->data;
  a->scales = base->scales;
  a->dtype = base->dtype;
  a->n = base->n;
  a->d = base->d;
  a->nbrs = graph->nbrs;
  a->R = graph->R;
  a->entry = graph->entry;
  a->nq = nq;
  a->k = P->k;
  a->ef = P->ef;
  a->test_mode = P->test_mode;
  a->routing = P->routing;
  a->hash_bits = hb;
  a->hash_min_bits = hb_min;
  a->wide = codes ? codes->wide : nullptr;
  a->max_exp = P->max_expansions > 0 ? P->max_expansions : (1 << 30);
  a->warps_per_cta = warps;
  a->entries = P->entries;
  const size_t per_warp =
      search_smem_per_warp(a->d, a->ef, hb, a->L, a->m, a->routing, a->R, a->perm != nullptr, a->beam);
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  while (warps > 1 && per_warp * warps > (size_t)maxsm) --warps;
  if (per_warp * warps > (size_t)maxsm)
    return set_error(PEOS_E_UNSUPPORTED, "per-query shared memory exceeds the per-CTA limit (lower ef or visited_slots)");
  a->warps_per_cta = warps;
  return PEOS_OK;
}

peos_status peos::attach_wide_flags(peos_codes_s* c, cudaStream_t st) {
  if (c->R <= 32) return PEOS_OK;
  uint8_t* w = nullptr;
  if (cudaMalloc(&w, (size_t)(c->n > 0 ? c->n : 1)) != cudaSuccess) return set_error(PEOS_E_NOMEM, "cudaMalloc wide");
  cudaError_t e = launch_wide_flags(c->records, c->rec_stride, rec_ids_offset(c->R, c->scalar_bits), c->n, c->R, w, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(w);
    return cuda_error(e, "second-group flags");
  }
  c->wide = w;
  return PEOS_OK;
}

extern "C" {

peos_status peos_search_rerank(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                               const peos_matrix* rerank, const peos_matrix* queries,
                               const peos_search_params* params, int32_t* ids_out, float* dists_out,
                               int32_t* counters, void* stream) {
  NvtxRange nvtx_range("peos.search");
  peos_status st = check_matrix(queries, "queries");
  if (st) return st;
  SearchLaunch a;
  st = prepare_search(graph, codes, base, queries->n, queries->d, params, &a);
  if (st) return st;
  st = check_rerank(rerank, base, a);
  if (st) return st;
  if (queries->n > 0 && (!ids_out || !dists_out)) return set_error(PEOS_E_INVAL, "NULL output");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  a.Q = static_cast<const float*>(queries->data);
  a.ids_out = ids_out;
  a.dists_out = dists_out;
  a.counters = counters;
  if (queries->n == 0) return PEOS_OK;
  StreamScratch work(s);
  const size_t tb = search_scratch_bytes(queries->n, a.L, a.m, a.routing);
  const size_t lb = rerank ? (size_t)queries->n * a.ef * sizeof(int32_t) : 0;
  const size_t o_t = 256, o_i = o_t + ((tb + 255) & ~(size_t)255), o_d = o_i + ((lb + 255) & ~(size_t)255);
  cudaError_t e = work.alloc(o_d + lb);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync");
  char* wp = static_cast<char*>(work.p);
  a.work = reinterpret_cast<int*>(wp);
  if (rerank) {
    a.Xr = static_cast<const float*>(rerank->data);
    a.rr_ids = reinterpret_cast<int32_t*>(wp + o_i);
    a.rr_dists = reinterpret_cast<float*>(wp + o_d);
  }
  e = launch_search(a, s);
  if (e != cudaSuccess) return cuda_error(e, "search launch");
  return PEOS_OK;
}

peos_status peos_search_batch_workspace_size(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                                             const peos_matrix* rerank, int64_t nq,
                                             const peos_search_params* params, size_t* bytes) {
  if (!bytes) return set_error(PEOS_E_INVAL, "bytes is NULL");
  SearchLaunch a;
  peos_status st = prepare_search(graph, codes, base, nq, base ? base->d : 0, params, &a);
  if (st) return st;
  st = check_rerank(rerank, base, a);
  if (st) return st;
  *bytes = batch_layout(a, nq, rerank != nullptr).total;
  return PEOS_OK;
}

peos_status peos_search_batch(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                              const peos_matrix* rerank, const peos_matrix* queries,
                              const peos_search_params* params, const int32_t* k_per_query,
                              const int32_t* ef_per_query, int32_t* ids_out, float* dists_out, int32_t* counters,
                              void* workspace, size_t workspace_bytes, void* stream) {
  NvtxRange nvtx_range("peos.search");
  peos_status st = check_matrix(queries, "queries");
  if (st) return st;
  SearchLaunch a;
  st = prepare_search(graph, codes, base, queries->n, queries->d, params, &a);
  if (st) return st;
  st = check_rerank(rerank, base, a);
  if (st) return st;
  if (queries->n > 0 && (!ids_out || !dists_out)) return set_error(PEOS_E_INVAL, "NULL output");
  const BatchLayout L = batch_layout(a, queries->n, rerank != nullptr);
  if (!workspace || ((uintptr_t)workspace & 255) != 0)
    return set_error(PEOS_E_INVAL, "workspace must be non-NULL and 256-byte aligned");
  if (workspace_bytes < L.total) return set_error(PEOS_E_INVAL, "workspace too small");
  char* w = static_cast<char*>(workspace);
  a.Q = static_cast<const float*>(queries->data);
  a.ids_out = ids_out;
  a.dists_out = dists_out;
  a.counters = counters;
  a.k_q = k_per_query;
  a.ef_q = ef_per_query;
  a.work = reinterpret_cast<int*>(w);
  a.order = reinterpret_cast<int32_t*>(w + L.order);
  if (rerank) {
    a.Xr = static_cast<const float*>(rerank->data);
    a.rr_ids = reinterpret_cast<int32_t*>(w + L.rr_ids);
    a.rr_dists = reinterpret_cast<float*>(w + L.rr_dists);
  }
  cudaError_t e = launch_search(a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "batch search launch");
  return PEOS_OK;
}

peos_status peos_search(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                        const peos_matrix* queries, const peos_search_params* params, int32_t* ids_out,
                        float* dists_out, int32_t* counters, void* stream) {
  NvtxRange nvtx_range("peos.search");
  return peos_search_rerank(graph, codes, base, nullptr, queries, params, ids_out, dists_out, counters, stream);
}

peos_status peos_quantize(const peos_matrix* src, int32_t dtype, void* data_out, float* scales_out, void* stream) {
  NvtxRange nvtx_range("peos.quantize");
  peos_status st = check_matrix(src, "src");
  if (st) return st;
  if (dtype != PEOS_BF16 && dtype != PEOS_FP8E4M3) return set_error(PEOS_E_INVAL, "dtype must be BF16 or FP8E4M3");
  if (src->n > 0 && !data_out) return set_error(PEOS_E_INVAL, "data_out is NULL");
  if (dtype == PEOS_FP8E4M3 && src->n > 0 && !scales_out) return set_error(PEOS_E_INVAL, "scales_out is NULL");
  cudaError_t e = launch_quantize(static_cast<const float*>(src->data), src->n, src->d, dtype, data_out, scales_out,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "quantize launch");
  return PEOS_OK;
}

static peos_status search_host_impl(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                                    const float* queries_host, int64_t nq, const peos_search_params* params,
                                    int32_t* ids_host, float* dists_host, int32_t* counters_host, void* stream,
                                    bool wait) {
  SearchLaunch a;
  peos_status st = prepare_search(graph, codes, base, nq, base ? base->d : 0, params, &a);
  if (st) return st;
  if (nq == 0) return PEOS_OK;
  if (!queries_host || !ids_host || !dists_host) return set_error(PEOS_E_INVAL, "NULL host buffer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t qb = (size_t)nq * a.d * sizeof(float);
  const size_t ib = (size_t)nq * a.k * sizeof(int32_t);
  const size_t db = (size_t)nq * a.k * sizeof(float);
  const size_t cb = counters_host ? (size_t)nq * PEOS_NCOUNTERS * sizeof(int32_t) : 0;
  const size_t tb = search_scratch_bytes(nq, a.L, a.m, a.routing);
  const size_t eb = a.entries ? (size_t)nq * sizeof(int32_t) : 0;  // host entries, copied in
  const size_t o_q = 0, o_i = (qb + 255) & ~(size_t)255, o_d = (o_i + ib + 255) & ~(size_t)255,
               o_c = (o_d + db + 255) & ~(size_t)255, o_w = (o_c + cb + 255) & ~(size_t)255, o_e = o_w + 256,
               o_t = (o_e + eb + 255) & ~(size_t)255;
  StreamScratch buf(s);
  cudaError_t e = buf.alloc(o_t + tb);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync");
  char* base_p = static_cast<char*>(buf.p);
  a.Q = reinterpret_cast<const float*>(base_p + o_q);
  a.ids_out = reinterpret_cast<int32_t*>(base_p + o_i);
  a.dists_out = reinterpret_cast<float*>(base_p + o_d);
  a.counters = counters_host ? reinterpret_cast<int32_t*>(base_p + o_c) : nullptr;
  a.work = reinterpret_cast<int*>(base_p + o_w);
  e = cudaMemcpyAsync(base_p + o_q, queries_host, qb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && a.entries) {
    e = cudaMemcpyAsync(base_p + o_e, a.entries, eb, cudaMemcpyHostToDevice, s);
    a.entries = reinterpret_cast<const int32_t*>(base_p + o_e);
  }
  if (e == cudaSuccess) e = launch_search(a, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ids_host, a.ids_out, ib, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dists_host, a.dists_out, db, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && counters_host) e = cudaMemcpyAsync(counters_host, a.counters, cb, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_error(e, "peos_search_host");
  if (wait) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "peos_search_host sync");
  }
  return PEOS_OK;  // without wait the staging area is released stream-ordered after the copies
}

peos_status peos_search_host(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                             const float* queries_host, int64_t nq, const peos_search_params* params, int32_t* ids_host,
                             float* dists_host, int32_t* counters_host, void* stream) {
  NvtxRange nvtx_range("peos.search");
  return search_host_impl(graph, codes, base, queries_host, nq, params, ids_host, dists_host, counters_host, stream,
                          true);
}

peos_status peos_search_host_async(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                                   const float* queries_host, int64_t nq, const peos_search_params* params,
                                   int32_t* ids_host, float* dists_host, int32_t* counters_host, void* stream) {
  NvtxRange nvtx_range("peos.search");
  return search_host_impl(graph, codes, base, queries_host, nq, params, ids_host, dists_host, counters_host, stream,
                          false);
}

peos_status peos_release_workspace(void) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceSynchronize");
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
  return PEOS_OK;
}

peos_status peos_edge_stats(peos_codes_t codes, const float* query, int32_t v, float dv, float delta2, float eps,
                            int32_t eta_mode, float* A_out, float* H_out, float* T_out, int32_t* pass_out,
                            int32_t* kind_out, void* stream) {
  NvtxRange nvtx_range("peos.edge_stats");
  if (!codes || !query || !A_out || !H_out || !T_out || !pass_out || !kind_out)
    return set_error(PEOS_E_INVAL, "NULL argument");
  if (v < 0 || (int64_t)v >= codes->n) return set_error(PEOS_E_INVAL, "v outside [0, n)");
  if (codes->kind != kCodesPeos) return set_error(PEOS_E_INVAL, "edge statistics need PEOs codes");
  if (codes->scalar_bits != 32)
    return set_error(PEOS_E_UNSUPPORTED, "edge statistics read FP32 scalars (codes with 8/16-bit scalars: search only)");
  if (!(eps > 0.0f && eps <= 0.5f)) return set_error(PEOS_E_INVAL, "eps must be in (0, 0.5]");
  if (eta_mode != 0 && eta_mode != 1) return set_error(PEOS_E_INVAL, "eta_mode must be 0 or 1");
  const float z = (float)norm_ppf((double)eps);
  const float c = (float)(sqrt((double)codes->L) * eta_value(codes->m, eta_mode));
  cudaError_t e = launch_edge_stats(codes, query, v, dv, delta2, z, c, A_out, H_out, T_out, pass_out, kind_out,
                                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "edge stats launch");
  return PEOS_OK;
}

peos_status peos_knn_tensor(const peos_matrix* base, const peos_matrix* queries, int32_t k, int32_t* ids_out,
                            float* dists_out, void* stream) {
  NvtxRange nvtx_range("peos.knn");
  peos_status st = check_matrix(base, "base");
  if (st) return st;
  st = check_matrix(queries, "queries");
  if (st) return st;
  if (queries->d != base->d) return set_error(PEOS_E_INVAL, "queries.d != base.d");
  if (k < 1 || k > knn_tc_max_k() || k > base->n)
    return set_error(PEOS_E_INVAL, "need 1 <= k <= min(96, n) for the tensor-core brute force");
  if (base->n > 0x7fffffffLL || queries->n > 0x7fffffffLL) return set_error(PEOS_E_INVAL, "too many rows");
  if (queries->n == 0) return PEOS_OK;
  if (!ids_out || !dists_out) return set_error(PEOS_E_INVAL, "NULL output");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  StreamScratch scratch(s);
  const size_t bytes = knn_tc_scratch_bytes(base->n, queries->n, base->d, k, sms);
  cudaError_t e = scratch.alloc(bytes + 256);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync");
  int* err = reinterpret_cast<int*>(static_cast<char*>(scratch.p) + bytes);
  e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = launch_knn_tc(static_cast<const float*>(base->data), base->n, base->d,
                      static_cast<const float*>(queries->data), queries->n, k, ids_out, dists_out, scratch.p, err, s);
  if (e == cudaErrorNotSupported) return set_error(PEOS_E_UNSUPPORTED, "tensor maps are not available");
  if (e != cudaSuccess) return cuda_error(e, "tensor-core brute force");
  int h = 0;
  e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "tensor-core brute force");
  if (h) return set_error(PEOS_E_TIMEOUT, "a tensor-core brute-force CTA gave up waiting for its tiles");
  return PEOS_OK;
}

peos_status peos_hier_entry(const peos_hierarchy* h, const peos_matrix* base, const peos_matrix* queries,
                            int32_t* entries, void* stream) {
  NvtxRange nvtx_range("peos.hier_entry");
  if (!h || !h->layers) return set_error(PEOS_E_INVAL, "hierarchy is NULL");
  peos_status st = check_matrix(base, "base", /*stored=*/true);
  if (st) return st;
  st = check_matrix(queries, "queries");
  if (st) return st;
  if (queries->d != base->d) return set_error(PEOS_E_INVAL, "queries.d != base.d");
  if (h->levels < 1 || h->levels > kMaxHierLevels) return set_error(PEOS_E_INVAL, "levels must be in 1..8");
  HierLaunch L{};
  L.levels = h->levels;
  L.top_entry = h->top_entry;
  for (int l = 0; l < h->levels; ++l) {
    const peos_layer& y = h->layers[l];
    if (y.n < 1 || y.n > INT32_MAX || y.R < 1 || y.R > 32 || !y.ids || !y.nbrs)
      return set_error(PEOS_E_INVAL, "layer " + std::to_string(l) + ": need n >= 1, 1 <= R <= 32, ids and nbrs");
    if (l + 1 < h->levels && !y.down) return set_error(PEOS_E_INVAL, "layer " + std::to_string(l) + ": down is NULL");
    L.n[l] = y.n;
    L.R[l] = y.R;
    L.ids[l] = y.ids;
    L.nbrs[l] = y.nbrs;
    L.down[l] = l + 1 < h->levels ? y.down : nullptr;
  }
  if (h->top_entry < 0 || h->top_entry >= h->layers[0].n) return set_error(PEOS_E_INVAL, "top_entry out of range");
  if (queries->n > 0 && !entries) return set_error(PEOS_E_INVAL, "entries is NULL");
  if (queries->n == 0) return PEOS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScratch work(s);
  cudaError_t e = work.alloc(256);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync");
  e = launch_hier_entry(L, base->data, base->scales, base->dtype, base->n, base->d,
                        static_cast<const float*>(queries->data), queries->n, static_cast<int*>(work.p), entries, s);
  if (e != cudaSuccess) return cuda_error(e, "hierarchical entry launch");
  return PEOS_OK;
}

peos_status peos_selftest_bounded_wait(int64_t limit_us, int32_t* gave_up, void* stream) {
  if (!gave_up) return set_error(PEOS_E_INVAL, "gave_up is NULL");
  if (limit_us < 1 || limit_us > 2000000) return set_error(PEOS_E_INVAL, "limit_us must be in 1..2000000");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScratch flag(s);
  cudaError_t e = flag.alloc(sizeof(int));
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync");
  int* d = static_cast<int*>(flag.p);
  e = cudaMemsetAsync(d, 0xff, sizeof(int), s);
  if (e == cudaSuccess) e = launch_bounded_wait_probe((long long)limit_us * 1000, d, s);
  int h = -1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "bounded-wait self-test");
  *gave_up = h;
  return PEOS_OK;
}

peos_status peos_knn_bruteforce(const peos_matrix* base, const peos_matrix* queries, int32_t k, int32_t* ids_out,
                                float* dists_out, void* stream) {
  NvtxRange nvtx_range("peos.knn");
  peos_status st = check_matrix(base, "base");
  if (st) return st;
  st = check_matrix(queries, "queries");
  if (st) return st;
  if (queries->d != base->d) return set_error(PEOS_E_INVAL, "queries.d != base.d");
  if (k < 1 || k > 256) return set_error(PEOS_E_INVAL, "k must be in 1..256");
  if (base->n < 1) return set_error(PEOS_E_INVAL, "empty base");
  if (queries->n > 0 && (!ids_out || !dists_out)) return set_error(PEOS_E_INVAL, "NULL output");
  if (queries->n == 0) return PEOS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the per-chunk lists take nq x chunks x k keys: the queries go in slices whose lists
  // fit in 1 GiB (at least 32 queries, one CTA's worth, per slice)
  const size_t per_query = knn_scratch_bytes(base->n, 1, k);
  int64_t slice = (int64_t)((size_t)1 << 30) / (int64_t)per_query;
  slice = slice < 32 ? 32 : slice - slice % 32;
  if (slice > queries->n) slice = queries->n;
  StreamScratch scratch(s);
  cudaError_t e = scratch.alloc(knn_scratch_bytes(base->n, slice, k));
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync knn scratch");
  const float* Q = static_cast<const float*>(queries->data);
  for (int64_t q0 = 0; q0 < queries->n; q0 += slice) {
    const int64_t nq = queries->n - q0 < slice ? queries->n - q0 : slice;
    e = launch_knn(static_cast<const float*>(base->data), base->n, base->d, Q + (size_t)q0 * base->d, nq, k,
                   ids_out + (size_t)q0 * k, dists_out + (size_t)q0 * k, scratch.p, s);
    if (e != cudaSuccess) return cuda_error(e, "knn launch");
  }
  return PEOS_OK;
}

}  // extern "C"
