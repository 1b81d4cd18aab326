// Batched graph search with PEOs routing (Algorithm 1 + Algorithm 2 of the paper),
// one warp per query, persistent CTAs pulling queries from a work counter.
//
// Per query, in the warp's slice of shared memory:
//   q      d floats                       the query
//   rd/ri  ef floats / ef ints            the result list R, sorted by (dist, id);
//                                         bit 31 of ri marks an expanded entry
//   vis    2^hash_bits ints               lossy visited table (see device.cuh)
//   tq/td  (L+1)m floats each             table of q, and of x = q - v for the node
//                                         being expanded (td = tq - node_proj[v])
//   cid    64 ints                        ids of the neighbours that passed
//   ckey   64 u64, cpos 64 ints           candidates kept for the merge, and
//                                         their insertion positions in R
//
// One expansion: pick the first unexpanded entry of R; read v's edge record (ids,
// ||e||, w_reg, codes) with coalesced loads, one edge per lane; drop visited heads;
// run the PEOs test per lane; gather the passing neighbours' vectors (float4 per
// lane, up to 8 rows in flight) and reduce their exact distances across the warp;
// sort the batch with a warp bitonic sort and merge it into R in place.
#include <cuda_runtime.h>
#include <math.h>

#include "device.cuh"
#include "internal.h"

namespace peos {

namespace {

constexpr int kGather = 8;  // candidate rows gathered concurrently per warp

struct Smem {
  float* q;
  float* rd;
  int32_t* ri;
  int32_t* vis;
  float* tq;
  float* td;
  int32_t* cid;
  uint64_t* ckey;
  int32_t* cpos;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t smem_layout(int d, int ef, int hash_bits, int L, int m, int routing,
                                              size_t* off /* 9 offsets or null */) {
  size_t o = 0;
  size_t offs[9];
  offs[0] = o; o = align16(o + (size_t)d * 4);
  offs[1] = o; o = align16(o + (size_t)ef * 4);
  offs[2] = o; o = align16(o + (size_t)ef * 4);
  offs[3] = o; o = align16(o + ((size_t)4 << hash_bits));
  const size_t tw = routing ? (size_t)(L + 1) * m : 0;
  offs[4] = o; o = align16(o + tw * 4);
  offs[5] = o; o = align16(o + tw * 4);
  offs[6] = o; o = align16(o + 64 * 4);
  offs[7] = o; o = align16(o + 64 * 8);
  offs[8] = o; o = align16(o + 64 * 4);
  if (off)
    for (int i = 0; i < 9; ++i) off[i] = offs[i];
  return o;
}

struct KArgs {
  const float* __restrict__ X;
  long long n;
  int d;
  const int32_t* __restrict__ nbrs;
  int R;
  int entry;
  const uint8_t* __restrict__ rec;
  size_t rec_stride;
  const float* __restrict__ tv;
  const float* __restrict__ A;
  const float* __restrict__ B;
  const float* __restrict__ Q;
  long long nq;
  int k, ef;
  int32_t* __restrict__ ids_out;
  float* __restrict__ dists_out;
  int32_t* __restrict__ counters;
  TestConst K;
  int hash_bits;
  int max_exp;
  int smem_per_warp;
  int* work;
};

// exact squared distances of up to kGather rows to the query, warp-cooperative
__device__ __forceinline__ void gather_dists(const float4* __restrict__ q4, const float* __restrict__ X, int d4,
                                             const int32_t* ids, int cnt, float* out, int lane) {
  float acc[kGather];
#pragma unroll
  for (int g = 0; g < kGather; ++g) acc[g] = 0.0f;
  for (int c = lane; c < d4; c += 32) {
    const float4 qv = q4[c];
    float4 u[kGather];
#pragma unroll
    for (int g = 0; g < kGather; ++g)
      if (g < cnt) u[g] = __ldg(reinterpret_cast<const float4*>(X + (size_t)ids[g] * (size_t)(d4 * 4)) + c);
#pragma unroll
    for (int g = 0; g < kGather; ++g) {
      if (g < cnt) {
        const float dx = qv.x - u[g].x, dy = qv.y - u[g].y, dz = qv.z - u[g].z, dw = qv.w - u[g].w;
        acc[g] = fmaf(dx, dx, acc[g]);
        acc[g] = fmaf(dy, dy, acc[g]);
        acc[g] = fmaf(dz, dz, acc[g]);
        acc[g] = fmaf(dw, dw, acc[g]);
      }
    }
  }
#pragma unroll
  for (int g = 0; g < kGather; ++g) out[g] = warp_sum(acc[g]);
}

template <int ROUTING, int NR>
__global__ void __launch_bounds__(512) search_kernel(KArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  size_t off[9];
  smem_layout(a.d, a.ef, a.hash_bits, a.K.L, a.K.m, ROUTING, off);
  unsigned char* base = smem_raw + (size_t)warp * a.smem_per_warp;
  Smem s;
  s.q = reinterpret_cast<float*>(base + off[0]);
  s.rd = reinterpret_cast<float*>(base + off[1]);
  s.ri = reinterpret_cast<int32_t*>(base + off[2]);
  s.vis = reinterpret_cast<int32_t*>(base + off[3]);
  s.tq = reinterpret_cast<float*>(base + off[4]);
  s.td = reinterpret_cast<float*>(base + off[5]);
  s.cid = reinterpret_cast<int32_t*>(base + off[6]);
  s.ckey = reinterpret_cast<uint64_t*>(base + off[7]);
  s.cpos = reinterpret_cast<int32_t*>(base + off[8]);

  const int d = a.d, d4 = d >> 2, R = a.R, ef = a.ef;
  const int hb = a.hash_bits;
  const int H = 1 << hb;
  const int tw = (a.K.L + 1) * a.K.m;
  const float4* q4 = reinterpret_cast<const float4*>(s.q);

  for (;;) {
    int qi = 0;
    if (lane == 0) qi = atomicAdd(a.work, 1);
    qi = __shfl_sync(kFull, qi, 0);
    if ((long long)qi >= a.nq) break;

    const float4* qg = reinterpret_cast<const float4*>(a.Q + (size_t)qi * d);
    for (int c = lane; c < d4; c += 32) reinterpret_cast<float4*>(s.q)[c] = __ldg(qg + c);
    for (int h = lane; h < H; h += 32) s.vis[h] = -1;
    __syncwarp();
    if (ROUTING) {
      project_table(s.q, d, a.K.L, a.K.m, a.A, a.B, s.tq, lane);
      __syncwarp();
    }

    int c_edges = 0, c_vskip = 0, c_arej = 0, c_aacc = 0, c_htest = 0, c_hpass = 0;  // per lane
    int c_exp = 0, c_full = 0, c_ndist = 0, c_ins = 0, status = PEOS_OK;           // warp-uniform

    {
      int32_t ids1[kGather];
      float dd[kGather];
      ids1[0] = a.entry;
      gather_dists(q4, a.X, d4, ids1, 1, dd, lane);
      if (lane == 0) {
        s.rd[0] = dd[0];
        s.ri[0] = a.entry;
        s.vis[visit_slot(a.entry, hb)] = a.entry;
      }
      c_ndist = 1;
    }
    int len = 1, hint = 0;
    __syncwarp();

    for (;;) {
      // ---- select the first unexpanded entry of R
      int sel = -1;
      for (int b = hint; b < len; b += 32) {
        const int i = b + lane;
        const bool un = (i < len) && !(s.ri[i] & kExpanded);
        const unsigned bal = __ballot_sync(kFull, un);
        if (bal) { sel = b + __ffs(bal) - 1; break; }
      }
      if (sel < 0) break;
      if (c_exp >= a.max_exp) { status = PEOS_E_OVERFLOW; break; }
      hint = sel;
      const int32_t v = s.ri[sel];
      const float dv = s.rd[sel];
      __syncwarp();
      if (lane == 0) s.ri[sel] = v | kExpanded;
      ++c_exp;
      const bool full = (len == ef);
      const float delta2 = full ? s.rd[ef - 1] : INFINITY;

      // ---- edge record
      int32_t id[NR];
      float en[NR], wr[NR];
      const uint8_t* rec = ROUTING ? a.rec + (size_t)v * a.rec_stride : nullptr;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int sl = r * 32 + lane;
        id[r] = -1;
        en[r] = 0.0f;
        wr[r] = 0.0f;
        if (sl < R) id[r] = ROUTING ? __ldg(reinterpret_cast<const int32_t*>(rec) + sl) : __ldg(a.nbrs + (size_t)v * R + sl);
        if ((long long)id[r] >= a.n) id[r] = -1;  // never read outside the base
      }
      const bool testing = ROUTING && full && a.K.mode != 2;
      c_full += full ? 1 : 0;
      if (testing) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const int sl = r * 32 + lane;
          if (sl < R) {
            en[r] = __ldg(reinterpret_cast<const float*>(rec + 4 * (size_t)R) + sl);
            wr[r] = __ldg(reinterpret_cast<const float*>(rec + 8 * (size_t)R) + sl);
          }
        }
        const float* tvv = a.tv + (size_t)v * tw;
        for (int e = lane; e < tw; e += 32) s.td[e] = s.tq[e] - __ldg(tvv + e);
        __syncwarp();
      }

      // ---- visited filter and routing test
      bool pass[NR];
      unsigned pm[NR];
      int npass = 0;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int sl = r * 32 + lane;
        bool cand = id[r] >= 0;
        c_edges += cand ? 1 : 0;
        if (cand && s.vis[visit_slot(id[r], hb)] == id[r]) {
          cand = false;
          ++c_vskip;
        }
        bool p = cand;
        if (testing && cand) {
          float Ao, Ho, To;
          const int8_t* cd = reinterpret_cast<const int8_t*>(rec + 12 * (size_t)R) + sl;
          const int kind = peos_edge_test(s.td, dv, delta2, cd, R, en[r], wr[r], a.K, p, Ao, Ho, To);
          c_arej += kind == kRejectA;
          c_aacc += kind == kAcceptA;
          if (kind == kDecidedH) {
            ++c_htest;
            c_hpass += p ? 1 : 0;
          }
        }
        pass[r] = p;
        pm[r] = __ballot_sync(kFull, p);
      }
      {
        int before = 0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (pass[r]) {
            s.vis[visit_slot(id[r], hb)] = id[r];
            s.cid[before + __popc(pm[r] & ((1u << lane) - 1u))] = id[r];
          }
          before += __popc(pm[r]);
        }
        npass = before;
      }
      __syncwarp();
      if (npass == 0) continue;

      // ---- exact distances of the passing neighbours
      float mydist[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) mydist[r] = INFINITY;
      for (int b = 0; b < npass; b += kGather) {
        const int cnt = min(kGather, npass - b);
        int32_t gid[kGather];
#pragma unroll
        for (int g = 0; g < kGather; ++g) gid[g] = s.cid[b + (g < cnt ? g : 0)];
        float dd[kGather];
        gather_dists(q4, a.X, d4, gid, cnt, dd, lane);
#pragma unroll
        for (int g = 0; g < kGather; ++g) {
          const int gi = b + g;
          if (g < cnt && (gi & 31) == lane) {
#pragma unroll
            for (int r = 0; r < NR; ++r)
              if ((gi >> 5) == r) mydist[r] = dd[g];
          }
        }
      }
      c_ndist += npass;

      // ---- sort the batch; drop what cannot enter a full list
      uint64_t key[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int g = r * 32 + lane;
        key[r] = kNoKey;
        if (g < npass && (!full || mydist[r] < delta2)) key[r] = pack_key(mydist[r], s.cid[g]);
      }
      warp_sort<NR>(key, lane);

      // ---- insertion positions; drop entries already in R (forgotten by the visited table)
      int nkeep = 0;
      {
        int before = 0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          bool keep = false;
          int pos = 0;
          if (key[r] != kNoKey) {
            const float kd = key_dist(key[r]);
            const int32_t kid = key_id(key[r]);
            int lo = 0, hi = len;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              const float md = s.rd[mid];
              const int32_t mi = s.ri[mid] & ~kExpanded;
              const bool less = (md < kd) || (md == kd && mi < kid);
              if (less) lo = mid + 1; else hi = mid;
            }
            pos = lo;
            keep = !(lo < len && s.rd[lo] == kd && (s.ri[lo] & ~kExpanded) == kid);
          }
          const unsigned km = __ballot_sync(kFull, keep);
          if (keep) {
            const int g = before + __popc(km & ((1u << lane) - 1u));
            s.ckey[g] = key[r];
            s.cpos[g] = pos;
          }
          before += __popc(km);
        }
        nkeep = before;
      }
      __syncwarp();
      if (nkeep == 0) continue;

      // ---- Algorithm 1's rule in sorted order: candidate g enters iff every
      //      candidate before it did and dist < the (ef-1-g)-th entry of R
      //      (entries past len count as +inf)
      int J = 0;
      {
        bool stop = false;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const int g = r * 32 + lane;
          bool ok = false;
          if (g < nkeep) {
            const int idx = ef - 1 - g;
            const float bound = idx < 0 ? -INFINITY : (idx < len ? s.rd[idx] : INFINITY);
            ok = key_dist(s.ckey[g]) < bound;
          }
          const unsigned om = __ballot_sync(kFull, ok);
          if (!stop) {
            const unsigned lead = ~om;  // first failing lane
            if (lead == 0) {
              J += 32;
            } else {
              J += __ffs(lead) - 1;
              stop = true;
            }
          }
        }
        if (J > nkeep) J = nkeep;
      }
      if (J == 0) continue;

      // ---- in-place merge: shift R's tail from the back, then write the new entries
      const int p0 = s.cpos[0];
      for (int top = len - 1; top >= p0; top -= 32) {
        const int i = top - lane;
        float dd = 0.0f;
        int32_t ii = 0;
        int ni = ef;
        if (i >= p0) {
          dd = s.rd[i];
          ii = s.ri[i];
          int lo = 0, hi = J;  // number of accepted candidates with cpos <= i
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s.cpos[mid] <= i) lo = mid + 1; else hi = mid;
          }
          ni = i + lo;
        }
        __syncwarp();
        if (i >= p0 && ni < ef) {
          s.rd[ni] = dd;
          s.ri[ni] = ii;
        }
        __syncwarp();
      }
      for (int g = lane; g < J; g += 32) {
        const int idx = s.cpos[g] + g;
        const uint64_t kk = s.ckey[g];
        s.rd[idx] = key_dist(kk);
        s.ri[idx] = key_id(kk);
      }
      len = min(ef, len + J);
      hint = min(hint, p0);
      c_ins += J;
      __syncwarp();
    }

    // ---- outputs
    for (int j = lane; j < a.k; j += 32) {
      const bool have = j < len;
      a.ids_out[(size_t)qi * a.k + j] = have ? (s.ri[j] & ~kExpanded) : -1;
      a.dists_out[(size_t)qi * a.k + j] = have ? s.rd[j] : INFINITY;
    }
    if (a.counters) {
      const int e = warp_isum(c_edges), vs = warp_isum(c_vskip), ar = warp_isum(c_arej), aa = warp_isum(c_aacc),
                ht = warp_isum(c_htest), hp = warp_isum(c_hpass);
      if (lane == 0) {
        int32_t* cnt = a.counters + (size_t)qi * PEOS_NCOUNTERS;
        cnt[PEOS_C_EXPANSIONS] = c_exp;
        cnt[PEOS_C_EDGES] = e;
        cnt[PEOS_C_VISITED_SKIP] = vs;
        cnt[PEOS_C_A_REJECT] = ar;
        cnt[PEOS_C_A_ACCEPT] = aa;
        cnt[PEOS_C_H_TESTS] = ht;
        cnt[PEOS_C_H_PASS] = hp;
        cnt[PEOS_C_NDIST] = c_ndist;
        cnt[PEOS_C_INSERTS] = c_ins;
        cnt[PEOS_C_STATUS] = status;
        cnt[PEOS_C_FULL_EXPANSIONS] = c_full;
      }
    }
    __syncwarp();
  }
}

// Statistics of every out-edge of one node (one warp), same device code as the search.
__global__ void edge_stats_kernel(const float* __restrict__ q, int d, const uint8_t* __restrict__ recs,
                                  size_t rec_stride, int R, const float* __restrict__ tv,
                                  const float* __restrict__ A, const float* __restrict__ B, TestConst K, int v,
                                  float dv, float delta2, float* A_out, float* H_out, float* T_out,
                                  int32_t* pass_out, int32_t* kind_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int tw = (K.L + 1) * K.m;
  float* xs = reinterpret_cast<float*>(smem_raw);
  float* tq = xs + d;
  float* td = tq + tw;
  for (int k = lane; k < d; k += 32) xs[k] = q[k];
  __syncwarp();
  project_table(xs, d, K.L, K.m, A, B, tq, lane);
  __syncwarp();
  const float* tvv = tv + (size_t)v * tw;
  for (int e = lane; e < tw; e += 32) td[e] = tq[e] - tvv[e];
  __syncwarp();
  const uint8_t* rec = recs + (size_t)v * rec_stride;
  for (int sl = lane; sl < R; sl += 32) {
    const int32_t u = reinterpret_cast<const int32_t*>(rec)[sl];
    float Ao = 0.0f, Ho = 0.0f, To = 0.0f;
    bool p = false;
    int kind = -1;
    if (u >= 0) {
      const float en = reinterpret_cast<const float*>(rec + 4 * (size_t)R)[sl];
      const float wr = reinterpret_cast<const float*>(rec + 8 * (size_t)R)[sl];
      const int8_t* cd = reinterpret_cast<const int8_t*>(rec + 12 * (size_t)R) + sl;
      kind = peos_edge_test(td, dv, delta2, cd, R, en, wr, K, p, Ao, Ho, To);
    }
    A_out[sl] = Ao;
    H_out[sl] = Ho;
    T_out[sl] = To;
    pass_out[sl] = p ? 1 : 0;
    kind_out[sl] = kind;
  }
}

template <int ROUTING, int NR>
cudaError_t launch_t(const KArgs& ka, int warps, size_t smem_total, cudaStream_t st) {
  auto fn = search_kernel<ROUTING, NR>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_total);
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem_total);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long want = (ka.nq + warps - 1) / warps;
  long long grid = (long long)sms * per_sm;
  if (grid > want) grid = want;
  if (grid < 1) grid = 1;
  fn<<<(unsigned)grid, warps * 32, smem_total, st>>>(ka);
  return cudaGetLastError();
}

}  // namespace

size_t search_smem_per_warp(int d, int ef, int hash_bits, int L, int m, int routing) {
  return smem_layout(d, ef, hash_bits, L, m, routing, nullptr);
}

cudaError_t launch_search(const SearchLaunch& a, cudaStream_t st) {
  KArgs ka;
  ka.X = a.X;
  ka.n = a.n;
  ka.d = a.d;
  ka.nbrs = a.nbrs;
  ka.R = a.R;
  ka.entry = a.entry;
  ka.rec = a.rec;
  ka.rec_stride = a.rec_stride;
  ka.tv = a.tv;
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
  ka.K.mode = a.test_mode;
  ka.hash_bits = a.hash_bits;
  ka.max_exp = a.max_exp;
  ka.work = a.work;
  const size_t per_warp = search_smem_per_warp(a.d, a.ef, a.hash_bits, ka.K.L, ka.K.m, a.routing);
  ka.smem_per_warp = (int)per_warp;
  const int warps = a.warps_per_cta;
  const size_t total = per_warp * warps;
  cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (a.nq == 0) return cudaSuccess;
  if (a.R <= 32) {
    return a.routing ? launch_t<1, 1>(ka, warps, total, st) : launch_t<0, 1>(ka, warps, total, st);
  }
  return a.routing ? launch_t<1, 2>(ka, warps, total, st) : launch_t<0, 2>(ka, warps, total, st);
}

cudaError_t launch_edge_stats(const peos_codes_s* c, const float* q, int v, float dv, float delta2, float z_eps,
                              float c_eta, float* A_out, float* H_out, float* T_out, int32_t* pass_out,
                              int32_t* kind_out, cudaStream_t st) {
  TestConst K;
  K.z_eps = z_eps;
  K.c_eta = c_eta;
  K.L = c->L;
  K.m = c->m;
  K.mode = 0;
  const size_t smem = ((size_t)c->d + 2 * (size_t)(c->L + 1) * c->m) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(edge_stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  edge_stats_kernel<<<1, 32, smem, st>>>(q, c->d, c->records, c->rec_stride, c->R, c->node_proj, c->A, c->B, K, v,
                                         dv, delta2, A_out, H_out, T_out, pass_out, kind_out);
  return cudaGetLastError();
}

}  // namespace peos
