// Host side of the batched search: the launcher (the batch order for uneven batches,
// the search kernel of the stored element type, then the optional FP32 re-rank), the
// edge-statistics kernel used by diagnostics, and the FP32 instantiation of the search
// kernel (the kernel itself is in search_kernel.cuh).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "device.cuh"
#include "internal.h"
#include "search_kernel.cuh"

namespace peos {

namespace {

using namespace sk;

// Statistics of every out-edge of one node (one warp), same device code as the search.
__global__ void edge_stats_kernel(const float* __restrict__ q, const int32_t* __restrict__ perm, int d,
                                  const uint8_t* __restrict__ recs,
                                  size_t rec_stride, int R, int nwords, int bits, int cpw,
                                  const float* __restrict__ A, const float* __restrict__ B, TestConst K, int v,
                                  float dv, float delta2, float* A_out, float* H_out, float* T_out,
                                  int32_t* pass_out, int32_t* kind_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  float* xs = reinterpret_cast<float*>(smem_raw);
  float* t = xs + d;
  float* tq = t + (K.L + 1) * K.m;  // sign-folded
  for (int k = lane; k < d; k += 32) xs[k] = q[perm ? perm[k] : k];  // the codes' coordinates
  __syncwarp();
  project_table(xs, d, K.L, K.m, A, B, t, lane);
  __syncwarp();
  fold_table(t, K.L, K.m, bits, tq, lane);
  __syncwarp();
  const uint8_t* rec = recs + (size_t)v * rec_stride;
  const float xn = sqrtf(dv);
  const float inv = 1.0f / xn;
  for (int sl = lane; sl < R; sl += 32) {
    const int32_t u = reinterpret_cast<const int32_t*>(rec + rec_ids_offset(R))[sl];
    float Ao = 0.0f, Ho = 0.0f, To = 0.0f;
    bool p = false;
    int kind = -1;
    if (u >= 0) {
      const float4 f = reinterpret_cast<const float4*>(rec)[sl];
      unsigned long long cw[kMaxCodeWords];
      const unsigned long long* cp = reinterpret_cast<const unsigned long long*>(rec + rec_codes_offset(R)) + sl;
#pragma unroll
      for (int w = 0; w < kMaxCodeWords; ++w) cw[w] = (w < nwords) ? cp[(size_t)w * R] : 0ull;
      kind = peos_edge_test<true>(tq, f.w, dv, xn, inv, delta2, cw, bits, cpw, f.x, f.y, f.z, K, p, Ao, Ho, To);
    }
    A_out[sl] = Ao;
    H_out[sl] = Ho;
    T_out[sl] = To;
    pass_out[sl] = p ? 1 : 0;
    kind_out[sl] = kind;
  }
}

// Exact FP32 re-rank of each query's final list R (the precision form of the search:
// the list was ranked by distances to reduced-precision rows).  One warp per query
// recomputes the squared distance of every listed node from the FP32 base (all rows
// prefetched into L2 first, then gathered 8 at a time), sorts the (dist, id) keys with a
// bitonic network in its slice of shared memory and writes the k smallest.
constexpr int kRerankWarps = 8;
__global__ void __launch_bounds__(kRerankWarps * 32) rerank_kernel(const float* __restrict__ Q, long long nq, int d,
                                                                   const float* __restrict__ Xr,
                                                                   const int32_t* __restrict__ cand, int ef,
                                                                   int per_warp, int k, const int32_t* __restrict__ k_q,
                                                                   const int32_t* __restrict__ ef_q,
                                                                   int32_t* __restrict__ ids_out,
                                                                   float* __restrict__ dists_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem_raw + (size_t)warp * per_warp;
  float* s_q = reinterpret_cast<float*>(base);
  uint64_t* s_key = reinterpret_cast<uint64_t*>(base + align16((size_t)d * 4));
  const int d4 = d >> 2;
  const int lines_per_row = (d * 4 + 127) >> 7;
  const float4* q4 = reinterpret_cast<const float4*>(s_q);
  for (long long qi = (long long)blockIdx.x * kRerankWarps + warp; qi < nq; qi += (long long)gridDim.x * kRerankWarps) {
    const int32_t* c = cand + (size_t)qi * ef;
    // the list holds its len valid ids first, then -1
    int len = 0;
    for (int b = 0; b < ef; b += 32) len += __popc(__ballot_sync(kFull, b + lane < ef && c[b + lane] >= 0));
    for (int t = lane; t < len * lines_per_row; t += 32) {
      const int rr = t / lines_per_row, l = t - rr * lines_per_row;
      prefetch_l2(reinterpret_cast<const char*>(Xr + (size_t)c[rr] * d) + ((size_t)l << 7));
    }
    const float4* qg = reinterpret_cast<const float4*>(Q + (size_t)qi * d);
    for (int i = lane; i < d4; i += 32) reinterpret_cast<float4*>(s_q)[i] = __ldg(qg + i);
    int P = 1;
    while (P < len) P <<= 1;
    for (int i = lane; i < P; i += 32) s_key[i] = kNoKey;
    __syncwarp();
    for (int b = 0; b < len; b += 8) {
      const int cnt = min(8, len - b);
      int32_t gid[8];
#pragma unroll
      for (int g = 0; g < 8; ++g) gid[g] = c[b + (g < cnt ? g : 0)];
      const float tot = gather_dists<8, kF32>(q4, Xr, nullptr, d4, gid, cnt, lane);
      // lanes 4g .. 4g+3 hold the total of row g
      const int g = lane >> 2;
      if ((lane & 3) == 0 && g < cnt) s_key[b + g] = pack_key(tot, c[b + g]);
    }
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = lane; i < (P >> 1); i += 32) {
          const int lo = 2 * i - (i & (stride - 1));
          const int hi = lo + stride;
          const uint64_t x = s_key[lo], y = s_key[hi];
          const bool up = (lo & size) == 0;
          if ((x > y) == up) {
            s_key[lo] = y;
            s_key[hi] = x;
          }
        }
        __syncwarp();
      }
    }
    // this query's k (uneven batches); an invalid k or efs gives an empty result
    int kq = k;
    if (k_q) {
      kq = __ldg(k_q + qi);
      const int eq = ef_q ? __ldg(ef_q + qi) : ef;
      if (kq < 1 || kq > k || kq > eq) kq = 0;
    }
    for (int j = lane; j < k; j += 32) {
      const uint64_t key = (j < len && j < kq) ? s_key[j] : kNoKey;
      ids_out[(size_t)qi * k + j] = key == kNoKey ? -1 : key_id(key);
      dists_out[(size_t)qi * k + j] = key == kNoKey ? INFINITY : key_dist(key);
    }
    __syncwarp();
  }
}

// Order of an uneven batch: queries by descending efs (the longest searches start
// first, so the persistent CTAs finish together).  One CTA: a histogram of efs in
// shared memory, a descending exclusive scan, then a scatter (order within one efs
// value is arbitrary: every query's result is independent of the order).
constexpr int kOrderThreads = 1024;
__global__ void __launch_bounds__(kOrderThreads) order_by_ef_kernel(const int32_t* __restrict__ ef_q, long long nq,
                                                                    int ef_max, int32_t* __restrict__ order) {
  __shared__ int hist[kMaxEf + 2];
  for (int i = threadIdx.x; i <= ef_max + 1; i += kOrderThreads) hist[i] = 0;
  __syncthreads();
  auto bin = [&](long long q) {
    const int e = __ldg(ef_q + q);
    return e < 0 ? 0 : (e > ef_max ? ef_max + 1 : e);  // out-of-range values: their own bins
  };
  for (long long q = threadIdx.x; q < nq; q += kOrderThreads) atomicAdd(&hist[bin(q)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int b = ef_max + 1; b >= 0; --b) {
      const int c = hist[b];
      hist[b] = run;
      run += c;
    }
  }
  __syncthreads();
  for (long long q = threadIdx.x; q < nq; q += kOrderThreads) order[atomicAdd(&hist[bin(q)], 1)] = (int32_t)q;
}

// Per-warp slice: the query (16-byte aligned for float4 stores) and the keys; the
// slice size is a multiple of 16 bytes so that every warp's query stays aligned.
size_t rerank_smem_per_warp(int d, int ef) {
  size_t P = 1;
  while (P < (size_t)ef) P <<= 1;
  return align16(align16((size_t)d * 4) + 8 * P);
}

}  // namespace

template cudaError_t sk::launch_search_typed<sk::kF32, 1>(const KArgs&, int, int, int, int, size_t, cudaStream_t);

// Per-query device scratch of a search: none (each warp builds its query's table in
// shared memory).  Kept as a function so the entry points size scratch in one place.
size_t search_scratch_bytes(int64_t nq, int L, int m, int routing) {
  (void)nq;
  (void)L;
  (void)m;
  (void)routing;
  return 0;
}

// floats of the per-query table in the warp's slice: the sign-folded projection table
// (PEOs), the K values S_i . q (SimHash, m = K), none (plain)
static int query_table_floats(int routing, int L, int m) {
  return routing == 1 ? folded_stride(L, m) : routing == 2 ? m : 0;
}

size_t search_smem_per_warp(int d, int ef, int hash_bits, int L, int m, int routing, int R, bool permuted, int beam) {
  return smem_layout(d, ef, hash_bits, query_table_floats(routing, L, m), 0, routing, permuted,
                     cand_capacity(beam, R), nullptr);
}

namespace {

// The stages of one search call; `mark(i)` is called before stage i runs and, with
// i = PEOS_NSTAGES, after the last one.
template <class Mark>
cudaError_t run_search(const SearchLaunch& a, cudaStream_t st, Mark&& mark) {
  KArgs ka;
  ka.X = a.X;
  ka.n = a.n;
  ka.d = a.d;
  ka.nbrs = a.nbrs;
  ka.R = a.R;
  ka.entry = a.entry;
  ka.rec = a.rec;
  ka.rec_stride = a.routing ? a.rec_stride : 0;
  ka.tv_stride = query_table_floats(a.routing, a.L, a.m);
  ka.A = a.A;
  ka.B = a.B;
  ka.Q = a.Q;
  ka.nq = a.nq;
  ka.k = a.k;
  ka.ef = a.ef;
  ka.ids_out = a.ids_out;
  ka.dists_out = a.dists_out;
  ka.counters = a.counters;
  ka.K.z_eps = a.z_eps;
  ka.K.c_eta = a.c_eta;
  ka.K.L = a.routing ? a.L : 1;
  ka.K.m = a.routing ? a.m : 1;
  ka.K.kL = (float)ka.K.L / ((float)ka.K.L + 1.0f);
  ka.K.mode = a.test_mode;
  ka.code_words = a.routing == 1 ? code_words(a.L, a.m) : a.routing == 2 ? a.sh_K / 64 : 0;
  ka.code_bits = a.routing == 1 ? code_bits(a.m) : 2;
  ka.codes_per_word = a.routing == 1 ? codes_per_word(a.m) : 1;
  ka.sh_K = a.routing == 2 ? a.sh_K : 0;
  ka.sh_tv = a.sh_tv;
  for (int i = 0; i <= kMaxSimHashBits; ++i) ka.sh_acrit[i] = a.sh_acrit[i];
  ka.max_exp = a.max_exp;
  ka.work = a.work;
  ka.Wt = a.Wt;
  ka.wt_smem = 0;
  ka.perm = a.routing ? a.perm : nullptr;
  ka.norms = a.norms;
  ka.wide = a.wide;
#ifdef PEOS_CHECKED
  ka.check = check_counters();
  if (!ka.check) return cudaErrorMemoryAllocation;
#endif
  // kernel variant: PEOs 1 (frame T), 3 (frame Q), 4 / 5 (the same with the permutation)
  int kernel_routing =
      a.routing == 1 ? (a.frame == 1 ? 3 : 1) + (ka.perm ? (a.frame == 1 ? 2 : 3) : 0) : a.routing;
  // the compact index (frame T, no permutation): 6 = 16-bit, 7 = 8-bit edge scalars
  if (a.routing == 1 && a.scalar_bits == 16) kernel_routing = 6;
  if (a.routing == 1 && a.scalar_bits == 8) kernel_routing = 7;
  ka.scales = a.scales;
  ka.k_q = a.k_q;
  ka.ef_q = a.ef_q;
  ka.order = a.ef_q ? a.order : nullptr;
  ka.entries = a.entries;
  if (a.Xr) {  // the search keeps its whole list for the re-rank
    ka.k = a.ef;
    ka.k_q = nullptr;
    ka.ids_out = a.rr_ids;
    ka.dists_out = a.rr_dists;
  }
  // Shared memory and resident CTAs.  The register-bound CTAs per SM of the launch shape
  // come from its launch bounds (Shape<G>::kMinCtas CTAs of kMaxWarps warps: 3 at 8 rows
  // per gather batch, 4 at 4); the shared-memory bound from the SM's capacity and the
  // per-CTA reservation.
  int dev = 0, maxsm = 0, sm_total = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sm_total, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int warps = a.warps_per_cta;
  const int g = a.gather ? a.gather : default_gather(a.routing);
  const int by_regs = (g == 8 ? Shape<8>::kMinCtas : Shape<4>::kMinCtas) * kMaxWarps / warps;
  auto ctas = [&](size_t t) { return (int)((size_t)sm_total / (t + (size_t)reserved)); };
  const size_t extra = a.routing == 2 ? align16((size_t)(kMaxSimHashBits + 1) * sizeof(float)) : 0;  // thresholds
  const int tws = query_table_floats(a.routing, a.L, a.m);
  const int ncand = cand_capacity(a.beam, a.R);
  int hb = a.hash_bits;
  if (a.hash_min_bits > 0) {
    // automatic visited table: when the warps' shared memory, not their registers, limits
    // the resident CTAs, halve the table (down to hash_min_bits) and keep the largest size
    // among those that give the most resident CTAs (at most the register bound); forgetting
    // a few more nodes costs less than a CTA
    auto resident = [&](int b) {
      return std::min(by_regs, ctas(smem_layout(a.d, a.ef, b, tws, 0, a.routing, ka.perm != nullptr, ncand,
                                                nullptr) * warps + extra));
    };
    int best = resident(hb);
    for (int b = hb - 1; b >= a.hash_min_bits && best < by_regs; --b) {
      const int r = resident(b);
      if (r > best) {
        best = r;
        hb = b;
      }
    }
  }
  ka.hash_bits = hb;
  size_t offs[kNumOff];
  const size_t per_warp = smem_layout(a.d, a.ef, hb, tws, 0, a.routing, ka.perm != nullptr, ncand, offs);
  for (int i = 0; i < kNumOff; ++i) ka.off[i] = (int)offs[i];
  ka.smem_per_warp = (int)per_warp;
  size_t total = per_warp * warps + extra;
  if (a.routing == 1 && a.m <= 16) {
    // stage the k-major vectors in the CTA's shared memory when they fit beside the warps
    // and cost no resident CTA: with the copy the CTAs per SM must still reach the
    // register bound or the count without it, whichever is lower
    const size_t wt = align16((size_t)2 * a.d * a.m * sizeof(float));
    if (wt <= 32 * 1024 && total + wt <= (size_t)maxsm && ctas(total + wt) >= std::min(by_regs, ctas(total))) {
      ka.wt_smem = (int)wt;
      total += wt;
    }
  }
  cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (a.nq == 0) return cudaSuccess;
  mark(PEOS_STAGE_SETUP);
  if (ka.order) {
    order_by_ef_kernel<<<1, kOrderThreads, 0, st>>>(a.ef_q, a.nq, a.ef, a.order);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  mark(PEOS_STAGE_SEARCH);
  // code words held per edge: one when every edge's codes fit a word (plain routing reads none)
  const bool cw1 = ka.code_words <= 1;
  constexpr int CW3 = kMaxCodeWords;
  if (a.beam == 1) {
    switch (a.dtype) {
      case kF32:
        e = cw1 ? launch_search_typed<kF32, 1>(ka, kernel_routing, a.R, a.gather, warps, total, st)
                : launch_search_typed<kF32, CW3>(ka, kernel_routing, a.R, a.gather, warps, total, st);
        break;
      case kBF16:
        e = cw1 ? launch_search_typed<kBF16, 1>(ka, kernel_routing, a.R, a.gather, warps, total, st)
                : launch_search_typed<kBF16, CW3>(ka, kernel_routing, a.R, a.gather, warps, total, st);
        break;
      case kE4M3:
        e = cw1 ? launch_search_typed<kE4M3, 1>(ka, kernel_routing, a.R, a.gather, warps, total, st)
                : launch_search_typed<kE4M3, CW3>(ka, kernel_routing, a.R, a.gather, warps, total, st);
        break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (a.dtype) {
      case kF32:
        e = cw1 ? launch_search_beam<kF32, 1>(ka, kernel_routing, a.R, a.gather, a.beam, warps, total, st)
                : launch_search_beam<kF32, CW3>(ka, kernel_routing, a.R, a.gather, a.beam, warps, total, st);
        break;
      case kBF16:
        e = cw1 ? launch_search_beam<kBF16, 1>(ka, kernel_routing, a.R, a.gather, a.beam, warps, total, st)
                : launch_search_beam<kBF16, CW3>(ka, kernel_routing, a.R, a.gather, a.beam, warps, total, st);
        break;
      case kE4M3:
        e = cw1 ? launch_search_beam<kE4M3, 1>(ka, kernel_routing, a.R, a.gather, a.beam, warps, total, st)
                : launch_search_beam<kE4M3, CW3>(ka, kernel_routing, a.R, a.gather, a.beam, warps, total, st);
        break;
      default: return cudaErrorInvalidValue;
    }
  }
  if (e != cudaSuccess) return e;
  mark(PEOS_STAGE_RERANK);
  if (a.Xr) {  // exact FP32 re-rank of the lists
    const size_t per = rerank_smem_per_warp(a.d, a.ef);
    const size_t smem = per * kRerankWarps;
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(rerank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rerank_kernel, kRerankWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = (a.nq + kRerankWarps - 1) / kRerankWarps;
    if (grid > (long long)sms * per_sm) grid = (long long)sms * per_sm;
    rerank_kernel<<<(unsigned)grid, kRerankWarps * 32, smem, st>>>(a.Q, a.nq, a.d, a.Xr, a.rr_ids, a.ef, (int)per,
                                                                    a.k, a.k_q, a.ef_q, a.ids_out, a.dists_out);
    e = cudaGetLastError();
  }
  mark(PEOS_NSTAGES);
  return e;
}

}  // namespace

static_assert(kChkKinds == PEOS_CHECK_KINDS, "violation kinds of the C ABI");

#ifdef PEOS_CHECKED
// The violation counters of a self-checked build: kChkKinds counters in the library's
// device image (zero when the image loads, on every device), so that no search call,
// the allocation-free one included, allocates for them.  Host code reaches them through
// the address looked up once per device, with that device current.
static __device__ unsigned long long g_check_counts[kChkKinds];

unsigned long long* check_counters() {
  static std::mutex mu;
  static unsigned long long* per_dev[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!per_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_check_counts) != cudaSuccess) return nullptr;
    per_dev[dev] = static_cast<unsigned long long*>(p);
  }
  return per_dev[dev];
}
#endif

cudaError_t launch_search(const SearchLaunch& a, cudaStream_t st) {
  TraceCall tc;
  if (!trace_begin(&tc)) return run_search(a, st, [](int) {});
  int next = 0;  // events recorded so far
  cudaError_t e = run_search(a, st, [&](int i) {
    for (; next <= i; ++next) cudaEventRecord(tc.ev[next], st);
  });
  for (; next <= PEOS_NSTAGES; ++next) cudaEventRecord(tc.ev[next], st);
  trace_end(tc);
  return e;
}

size_t search_rerank_smem(int d, int ef) { return rerank_smem_per_warp(d, ef) * kRerankWarps; }

cudaError_t launch_edge_stats(const peos_codes_s* c, const float* q, int v, float dv, float delta2, float z_eps,
                              float c_eta, float* A_out, float* H_out, float* T_out, int32_t* pass_out,
                              int32_t* kind_out, cudaStream_t st) {
  TestConst K;
  K.z_eps = z_eps;
  K.c_eta = c_eta;
  K.L = c->L;
  K.m = c->m;
  K.kL = (float)c->L / ((float)c->L + 1.0f);
  K.mode = 0;
  const size_t smem =
      ((size_t)c->d + (size_t)(c->L + 1) * c->m + (size_t)folded_stride(c->L, c->m)) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(edge_stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  edge_stats_kernel<<<1, 32, smem, st>>>(q, c->perm, c->d, c->records, c->rec_stride, c->R, code_words(c->L, c->m),
                                         code_bits(c->m), codes_per_word(c->m), c->A, c->B, K, v, dv, delta2,
                                         A_out, H_out, T_out, pass_out, kind_out);
  return cudaGetLastError();
}

}  // namespace peos
