// The batched search kernel (Algorithm 1 + Algorithm 2 of the paper), templated on the
// element type of the stored base vectors so that each type compiles in its own
// translation unit: search.cu (FP32), search_bf16.cu, search_e4m3.cu.
//
// One warp per query, persistent CTAs pulling queries from a work counter.
// Per query, in the warp's slice of shared memory:
//   q      d floats                       the query (always FP32)
//   rd/ri  ef floats / ef ints            the result list R, sorted by (dist, id);
//                                         bit 31 of ri marks an expanded entry
//   vis    2^hash_bits ints               lossy visited table (see device.cuh)
//   tq     folded_stride floats           sign-folded projection table of q, built by the
//                                         warp when it takes the query
//   cid    64 ints                        ids of the neighbours that passed
//   ckey   64 u64, cpos 64 ints           candidates kept for the merge, and
//                                         their insertion positions in R
//
// One expansion: pick the first unexpanded entry of R; when the test will run, every
// lane loads its own edge's id, scalars (including the edge's node term of the
// statistic) and packed codes into registers (a single round trip); drop visited heads; run the PEOs test, one edge per lane; prefetch every passing
// neighbour's row into L2 and gather them G rows at a time (4 elements per lane per
// step), reducing the exact distances across the warp; rank the kept candidates and
// merge them into R in place.
//
// Reduced-precision storage: rows of BF16 (unscaled) or FP8 E4M3 with one FP32 scale
// per row; each element is widened exactly to FP32 and (E4M3) multiplied by its row's
// scale, and the distance accumulates in FP32.
#pragma once
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <math.h>

#include "device.cuh"
#include "internal.h"

namespace peos {
namespace sk {

// Launch shapes: G rows gathered per batch.  G = 8 runs within 80 registers (3 CTAs
// of 8 warps per SM), G = 4 within 64 registers (4 CTAs per SM).  Measured on GB300
// (1M x 128 FP32, R = 32): plain routing is fastest with G = 8, the PEOs kernel, which
// keeps more state live, with G = 4; these are the defaults, and a caller (the batch
// autotuner) can pick either.
constexpr int kMaxWarps = 8;  // warps (queries) per CTA
template <int G>
struct Shape {
  static_assert(G == 8 || G == 4, "gather_dists reduces 4 or 8 rows");
  static constexpr int kGather = G;
  static constexpr int kMinCtas = G == 8 ? 3 : 4;
};
__host__ __device__ constexpr int default_gather(int routing) { return routing ? 4 : 8; }

enum { kOffQ = 0, kOffRd, kOffRi, kOffVis, kOffTq, kOffCid, kOffCkey, kOffCpos, kOffQp, kNumOff };

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Candidates of one iteration (the passes of its W nodes): up to W * 32 * NR, at least 64.
__host__ __device__ inline int cand_capacity(int beam, int R) { return max(64, beam * (R <= 32 ? 32 : 64)); }

__host__ __device__ inline size_t smem_layout(int d, int ef, int hash_bits, int tws, size_t rec_stride,
                                              int routing, bool permuted, int ncand,
                                              size_t* off /* kNumOff offsets or null */) {
  size_t o = 0;
  size_t offs[kNumOff];
  offs[kOffQ] = o; o = align16(o + (size_t)d * 4);
  offs[kOffRd] = o; o = align16(o + (size_t)ef * 4);
  offs[kOffRi] = o; o = align16(o + (size_t)ef * 4);
  offs[kOffVis] = o; o = align16(o + ((size_t)4 << hash_bits));
  const size_t tb = routing ? (size_t)tws * 4 : 0;
  offs[kOffTq] = o; o = align16(o + tb);
  offs[kOffCid] = o; o = align16(o + (size_t)ncand * 4);
  offs[kOffCkey] = o; o = align16(o + (size_t)ncand * 8);
  offs[kOffCpos] = o; o = align16(o + (size_t)ncand * 4);
  // the query in the codes' permuted coordinates, read only by the table build: in the
  // candidate arrays (free while the table is built) when it fits there, else its own
  if (routing && permuted && (size_t)d * 4 <= offs[kOffCpos] + (size_t)ncand * 4 - offs[kOffCid]) {
    offs[kOffQp] = offs[kOffCid];
  } else {
    offs[kOffQp] = o; o = align16(o + (routing && permuted ? (size_t)d * 4 : 0));
  }
  if (off)
    for (int i = 0; i < kNumOff; ++i) off[i] = offs[i];
  return o;
}

struct KArgs {
  const void* __restrict__ X;  // n rows of d elements of the stored type
  long long n;
  int d;
  const int32_t* __restrict__ nbrs;
  int R;
  int entry;
  const uint8_t* __restrict__ rec;
  size_t rec_stride;
  int tv_stride;  // floats per (sign-folded) query projection table
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
  int off[kNumOff];  // per-warp shared-memory layout (bytes), computed on the host
  int* work;
  const float* __restrict__ Wt;       // k-major copy of the random vectors (PEOs)
  int wt_smem;                        // bytes at the start of shared memory holding Wt (0: read Wt from global)
  int code_words;                     // 64-bit code words per edge
  int code_bits;                      // bits per packed code
  int codes_per_word;                 // packed codes per 64-bit word
  const float* __restrict__ scales;   // FP8 E4M3 storage: per-row scale (else unused)
  const int32_t* __restrict__ perm;   // dimension permutation of the codes (PEOs), else null
  const int32_t* __restrict__ k_q;    // per-query k (uneven batches), else null (k for all)
  const int32_t* __restrict__ ef_q;   // per-query efs, else null (ef for all); ef is then the maximum
  const int32_t* __restrict__ order;  // order in which queries are taken from the work counter, or null
  const int32_t* __restrict__ entries;  // per-query entry nodes (hierarchical entry), or null (entry)
  // PEOs in frame Q (ROUTING = 3): squared norms of the base rows
  const float* __restrict__ norms;
  // R > 32: per node, 1 if it has an edge in slots 32..R-1 (from the index), or null
  const uint8_t* __restrict__ wide;
  // SimHash routing (ROUTING = 2): K bits, node table S_i . v (n x K), thresholds
  int sh_K;
  const float* __restrict__ sh_tv;
  float sh_acrit[kMaxSimHashBits + 1];
#ifdef PEOS_CHECKED
  unsigned long long* check;  // violation counters (kChk* kinds), checked builds only
#endif
};

// Self-checked builds (-DPEOS_CHECKED): every index the search computes into its list,
// its candidate arrays and the base is checked before use, and after every merge the list
// is checked to be strictly ascending in (dist, id) with no id twice.  A violation is
// counted by kind (read back with peos_check_read) and the access is skipped, so a bug
// shows up as a count, never as a fault.  Normal builds compile every check away.
#ifdef PEOS_CHECKED
#define PEOS_EXPECT(cond, kind) (expect_or_count((cond), a.check, (kind)))
__device__ __forceinline__ bool expect_or_count(bool ok, unsigned long long* c, int kind) {
  if (!ok) atomicAdd(c + kind, 1ull);
  return ok;
}
#else
#define PEOS_EXPECT(cond, kind) (true)
#endif

// Stored element types (the values of peos_dtype).
enum : int { kF32 = PEOS_F32, kBF16 = PEOS_BF16, kE4M3 = PEOS_FP8E4M3 };

// Four consecutive elements of a row, as loaded: 16, 8 or 4 bytes.
template <int DT> struct Row4;
template <> struct Row4<kF32> { using T = float4; static constexpr int kBytes = 4; };
template <> struct Row4<kBF16> { using T = uint2; static constexpr int kBytes = 2; };
template <> struct Row4<kE4M3> { using T = unsigned; static constexpr int kBytes = 1; };

// Elements 4c .. 4c+3 of row `id` (rows of 4*d4 elements).
template <int DT>
__device__ __forceinline__ typename Row4<DT>::T load_row4(const void* X, int32_t id, int d4, int c) {
  return __ldg(reinterpret_cast<const typename Row4<DT>::T*>(X) + (size_t)id * (size_t)d4 + c);
}

// Widen to FP32 (exact for both narrow types) and apply the row scale (E4M3).  The
// lower-addressed element sits in the lower bits of the loaded word.
__device__ __forceinline__ float4 widen4(float4 r, float) { return r; }
__device__ __forceinline__ float4 widen4(uint2 r, float) {
  return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u), __uint_as_float(r.y << 16),
                     __uint_as_float(r.y & 0xffff0000u));
}
__device__ __forceinline__ float4 widen4(unsigned r, float s) {
  const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(r & 0xffffu), __NV_E4M3);
  const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(r >> 16), __NV_E4M3);
  __half_raw h;
  h.x = lo.x;
  const float v0 = __half2float(__half(h));
  h.x = lo.y;
  const float v1 = __half2float(__half(h));
  h.x = hi.x;
  const float v2 = __half2float(__half(h));
  h.x = hi.y;
  const float v3 = __half2float(__half(h));
  return make_float4(s * v0, s * v1, s * v2, s * v3);
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Exact squared distances of up to G (4 or 8) rows to the query, warp-cooperative:
// each lane accumulates its float4 slices of every row, then a reduce-scatter
// (G/2 + ... + 1 shuffles, then plain xor steps) leaves the total of row g on the
// lanes whose top bits spell g; row_lane<G>(g) names one of them.
template <int G>
__device__ __forceinline__ int row_lane(int g) {
  if (G == 8) return ((g & 4) << 2) | ((g & 2) << 2) | ((g & 1) << 2);
  return ((g & 2) << 3) | ((g & 1) << 3);
}

template <int G, int DT>
__device__ __forceinline__ float gather_dists(const float4* __restrict__ q4, const void* __restrict__ X,
                                              const float* __restrict__ scales, int d4, const int32_t* ids, int cnt,
                                              int lane) {
  float acc[G], sc[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    acc[g] = 0.0f;
    sc[g] = 1.0f;
    if (DT == kE4M3 && g < cnt) sc[g] = __ldg(scales + ids[g]);
  }
  for (int c = lane; c < d4; c += 32) {
    const float4 qv = q4[c];
    typename Row4<DT>::T raw[G];
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < cnt) raw[g] = load_row4<DT>(X, ids[g], d4, c);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (g < cnt) {
        const float4 u = widen4(raw[g], sc[g]);
        const float dx = qv.x - u.x, dy = qv.y - u.y, dz = qv.z - u.z, dw = qv.w - u.w;
        acc[g] = fmaf(dx, dx, acc[g]);
        acc[g] = fmaf(dy, dy, acc[g]);
        acc[g] = fmaf(dz, dz, acc[g]);
        acc[g] = fmaf(dw, dw, acc[g]);
      }
    }
  }
  float a4[4];
  if (G == 8) {
    // 8 values -> 4 (xor 16): upper half-warp keeps rows 4..7, lower half rows 0..3
    const bool hi16 = lane & 16;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float keep = hi16 ? acc[(j + 4) % G] : acc[j % G];
      const float give = hi16 ? acc[j % G] : acc[(j + 4) % G];
      a4[j] = keep + __shfl_xor_sync(kFull, give, 16);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) a4[j] = acc[j % G];
  }
  // 4 -> 2 (xor 8 for G = 8, xor 16 for G = 4)
  const int o2 = (G == 8) ? 8 : 16;
  const bool hi2 = lane & o2;
  float a2[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float keep = hi2 ? a4[j + 2] : a4[j];
    const float give = hi2 ? a4[j] : a4[j + 2];
    a2[j] = keep + __shfl_xor_sync(kFull, give, o2);
  }
  // 2 -> 1 (xor 4 for G = 8, xor 8 for G = 4)
  const int o1 = (G == 8) ? 4 : 8;
  const bool hi1 = lane & o1;
  float a1 = (hi1 ? a2[1] : a2[0]) + __shfl_xor_sync(kFull, hi1 ? a2[0] : a2[1], o1);
  if (G == 4) a1 += __shfl_xor_sync(kFull, a1, 4);
  a1 += __shfl_xor_sync(kFull, a1, 2);
  a1 += __shfl_xor_sync(kFull, a1, 1);
  return a1;
}

// Distances of the passing rows b .. b+cnt-1 (cnt <= G): candidate i lives on lane i & 31
// of register i >> 5.
template <int G, int NR, int DT>
__device__ __forceinline__ void gather_batch(const float4* __restrict__ q4, const void* __restrict__ X,
                                             const float* __restrict__ scales, int d4, const int32_t* s_cid, int b,
                                             int cnt, int lane, float (&mydist)[NR]) {
  int32_t gid[G];
#pragma unroll
  for (int g = 0; g < G; ++g) gid[g] = s_cid[b + (g < cnt ? g : 0)];
  const float tot = gather_dists<G, DT>(q4, X, scales, d4, gid, cnt, lane);
  const int g = (lane - b) & 31;
  const float mine = __shfl_sync(kFull, tot, row_lane<G>(g & (G - 1)));
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int gi = r * 32 + lane;
    if (gi >= b && gi < b + cnt) mydist[r] = mine;
  }
}

#ifdef PEOS_CHECKED
// The list invariant after a merge: strictly ascending (dist, id), no id twice.
static __device__ __noinline__ void check_list(const float* s_rd, const int32_t* s_ri, int len, int lane,
                                        unsigned long long* c) {
  for (int i = lane; i + 1 < len; i += 32) {
    const float d0 = s_rd[i], d1 = s_rd[i + 1];
    const int32_t i0 = s_ri[i] & ~kExpanded, i1 = s_ri[i + 1] & ~kExpanded;
    if (!((d0 < d1) || (d0 == d1 && i0 < i1))) atomicAdd(c + kChkOrder, 1ull);
  }
  for (int i = lane; i < len; i += 32) {
    const int32_t x = s_ri[i] & ~kExpanded;
    for (int j = i + 1; j < len; ++j)
      if ((s_ri[j] & ~kExpanded) == x) atomicAdd(c + kChkDuplicate, 1ull);
  }
  __syncwarp();
}
#endif

// W = beam width: nodes expanded per iteration (1, 2 or 4); CW = 64-bit code words held
// per edge in registers (1 when every edge's L + 1 codes fit one word, else
// kMaxCodeWords; plain routing reads no codes and takes 1); QG: the query is read from
// global memory (long rows, when its shared-memory copy is what limits the resident CTAs),
// else from the warp's shared memory.
template <int ROUTING, int NR, bool COUNT, int DT, int G, int W, int CW, bool QG>
__global__ void __launch_bounds__(kMaxWarps * 32, Shape<G>::kMinCtas) search_kernel(KArgs a) {
  constexpr int kGather = Shape<G>::kGather;
  // NR = 2 (out-degree 33..64): a routing test with W = 1 holds one edge per lane and walks
  // two groups of 32 edges (the second only for a node that has an edge there: the test's
  // per-edge registers would otherwise spill); plain routing and W > 1 hold two edges per
  // lane (measured faster for them)
  constexpr bool kGroups = (NR == 2 && W == 1 && ROUTING != 0);
  constexpr int NL = kGroups ? 1 : NR;  // edges held per lane
  constexpr int NRC = W * NL;     // candidate registers per lane: candidate g = r * 32 + lane
  [[maybe_unused]] constexpr int kCand = NRC * 32;  // candidates one iteration can hold (checked builds)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // the CTA's copy of the k-major random vectors, read by every query's table build; it
  // sits after the warps' slices so that each slice starts at a multiple of its size
  const float* wt = a.Wt;
  float* s_acrit = nullptr;  // SimHash thresholds, staged after the warps' slices
  if (ROUTING == 2) {
    s_acrit = reinterpret_cast<float*>(smem_raw + (size_t)(blockDim.x >> 5) * a.smem_per_warp);
    for (int i = threadIdx.x; i <= a.sh_K; i += blockDim.x) s_acrit[i] = a.sh_acrit[i];
    __syncthreads();
  }
  // ROUTING: 0 plain, 2 SimHash; PEOs codes: 1 frame T, 3 frame Q, 4 frame T with the
  // dimension permutation, 5 frame Q with it, 6 / 7 frame T over 16- / 8-bit scalars
  constexpr bool kPeos = ROUTING == 1 || ROUTING >= 3;
  constexpr int kSB = ROUTING == 6 ? 16 : ROUTING == 7 ? 8 : 32;  // record scalar width
  constexpr bool kFrameQ = ROUTING == 3 || ROUTING == 5;
  constexpr bool kPerm = ROUTING == 4 || ROUTING == 5;
  if (kPeos && a.wt_smem) {
    unsigned char* tail = smem_raw + (size_t)(blockDim.x >> 5) * a.smem_per_warp;
    float4* dst = reinterpret_cast<float4*>(tail);
    const float4* src = reinterpret_cast<const float4*>(a.Wt);
    const int n4 = (2 * a.d * a.K.m) >> 2;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    wt = reinterpret_cast<const float*>(tail);
  }
  unsigned char* base = smem_raw + warp * a.smem_per_warp;
  float* s_q = reinterpret_cast<float*>(base + a.off[kOffQ]);  // the query (unless QG)
  float* s_rd = reinterpret_cast<float*>(base + a.off[kOffRd]);
  int32_t* s_ri = reinterpret_cast<int32_t*>(base + a.off[kOffRi]);
  int32_t* s_vis = reinterpret_cast<int32_t*>(base + a.off[kOffVis]);
  float* s_tq = reinterpret_cast<float*>(base + a.off[kOffTq]);
  int32_t* s_cid = reinterpret_cast<int32_t*>(base + a.off[kOffCid]);
  uint64_t* s_ckey = reinterpret_cast<uint64_t*>(base + a.off[kOffCkey]);
  int32_t* s_cpos = reinterpret_cast<int32_t*>(base + a.off[kOffCpos]);

  const int d = a.d, d4 = d >> 2, R = a.R;
  const int hb = a.hash_bits;
  const int H = 1 << hb;
  const int row_bytes = d * Row4<DT>::kBytes;
  const int lines_per_row = (row_bytes + 127) >> 7;
  // prefetch mapping, fixed for the kernel: with rows of up to 32 lines, lane l covers
  // line (l % lines_per_row) of every (32 / lines_per_row)-th row; longer rows take all
  // lanes per row
  const int pf_rows = lines_per_row <= 32 ? 32 / lines_per_row : 1;
  const int pf_row = lines_per_row <= 32 ? lane / lines_per_row : 0;
  const int pf_line = lines_per_row <= 32 ? lane - pf_row * lines_per_row : lane;

  for (;;) {
    int slot = 0;
    if (lane == 0) slot = atomicAdd(a.work, 1);
    slot = __shfl_sync(kFull, slot, 0);
    if ((long long)slot >= a.nq) break;
    const int qi = a.order ? __ldg(a.order + slot) : slot;

    // this query's list size and result count (uneven batches); out-of-range values
    // give an empty result and PEOS_E_INVAL in the query's status counter
    int ef = a.ef, kq = a.k, entry = a.entry;
    bool bad = false;
    if (a.entries) {
      entry = __ldg(a.entries + qi);
      bad = entry < 0 || (long long)entry >= a.n;
    }
    if (a.ef_q) {
      ef = __ldg(a.ef_q + qi);
      bad = bad || ef < 1 || ef > a.ef;
    }
    if (a.k_q) {
      kq = __ldg(a.k_q + qi);
      bad = bad || kq < 1 || kq > a.k || kq > ef;
    }
    if (bad) {
      for (int j = lane; j < a.k; j += 32) {
        a.ids_out[(size_t)qi * a.k + j] = -1;
        a.dists_out[(size_t)qi * a.k + j] = INFINITY;
      }
      if (COUNT && lane < PEOS_NCOUNTERS)
        a.counters[(size_t)qi * PEOS_NCOUNTERS + lane] = lane == PEOS_C_STATUS ? PEOS_E_INVAL : 0;
      continue;
    }

    const float4* qg = reinterpret_cast<const float4*>(a.Q + (size_t)qi * d);
    if (!QG)
      for (int c = lane; c < d4; c += 32) reinterpret_cast<float4*>(s_q)[c] = __ldg(qg + c);
    const float* qp = QG ? a.Q + (size_t)qi * d : s_q;  // the query, wherever it is read from
    const float4* q4 = reinterpret_cast<const float4*>(qp);
    for (int h = lane; h < H; h += 32) s_vis[h] = -1;
    __syncwarp();
    if (ROUTING == 2) {
      // SimHash: S_i . q, sequential sums (the bits of x = q - v come from it and S_i . v)
      for (int i = lane; i < a.sh_K; i += 32) {
        const float* si = a.B + (size_t)i * d;
        float acc = 0.0f;
        for (int k = 0; k < d; ++k) acc = acc + __ldg(si + k) * qp[k];
        s_tq[i] = acc;
      }
      __syncwarp();
    }
    float qq = 0.0f, qn = 0.0f;  // frame Q: ||q||^2 (sequential, one lane) and ||q||
    if (kPeos) {
      // the query's projection table (Algorithm 2's T_I for this query), sign-folded, of
      // the query in the codes' coordinates (Appendix D.1's permutation, when there is one)
      const float* s_qt = qp;
      if (kPerm) {
        float* s_qp = reinterpret_cast<float*>(base + a.off[kOffQp]);
        for (int t = lane; t < d; t += 32) s_qp[t] = qp[__ldg(a.perm + t)];
        __syncwarp();
        s_qt = s_qp;
      }
      if (a.K.m <= 16)
        project_table_folded_kmajor(s_qt, d, a.K.L, a.K.m, a.code_bits, wt, s_tq, lane);
      else
        project_table_folded(s_qt, d, a.K.L, a.K.m, a.code_bits, a.A, a.B, s_tq, lane);
      __syncwarp();
      if (kFrameQ) {
        // frame Q: the table of q' = q / ||q||
        if (lane == 0)
          for (int k = 0; k < d; ++k) qq = qq + qp[k] * qp[k];
        qq = __shfl_sync(kFull, qq, 0);
        qn = sqrtf(qq);
        if (qn > 0.0f) {
          const float iq = 1.0f / qn;
          for (int t = lane; t < a.tv_stride; t += 32) s_tq[t] = s_tq[t] * iq;
        }
        __syncwarp();
      }
    }

    int c_edges = 0, c_vskip = 0, c_arej = 0, c_aacc = 0, c_htest = 0, c_hpass = 0;  // per lane
    int c_exp = 0, c_full = 0, c_ndist = 0, c_ins = 0, status = PEOS_OK;           // warp-uniform

    {
      int32_t ids1[kGather];
      ids1[0] = entry;
      const float d0 = __shfl_sync(kFull, gather_dists<4, DT>(q4, a.X, a.scales, d4, ids1, 1, lane), row_lane<4>(0));
      if (lane == 0) {
        s_rd[0] = d0;
        s_ri[0] = entry;
        visit_mark(s_vis, entry, hb);
      }
      c_ndist = 1;
    }
    int len = 1, hint = 0;
    __syncwarp();

    for (;;) {
      // ---- select the W first unexpanded entries of R (the W smallest unexpanded (dist, id)).
      //      W = 1: every lane holds the node; W > 1: lane w holds node w of the iteration.
      int nsel = 0;
      int my_pos = -1;
      if constexpr (W == 1) {
        for (int b = hint; b < len; b += 32) {
          const int i = b + lane;
          const bool un = (i < len) && !(s_ri[i] & kExpanded);
          const unsigned bal = __ballot_sync(kFull, un);
          if (bal) {
            my_pos = b + __ffs(bal) - 1;
            nsel = 1;
            break;
          }
        }
      } else {
        for (int b = hint; b < len && nsel < W; b += 32) {
          const int i = b + lane;
          const bool un = (i < len) && !(s_ri[i] & kExpanded);
          const unsigned bal = __ballot_sync(kFull, un);
          if (bal == 0) continue;
          const int take = min(W - nsel, __popc(bal));
          // lanes nsel .. nsel + take - 1 fetch the positions of the first `take` set bits
          const bool recv = lane >= nsel && lane < nsel + take;
          const int src = recv ? (int)__fns(bal, 0, lane - nsel + 1) : 0;
          const int got = __shfl_sync(kFull, i, src);
          if (recv) my_pos = got;
          nsel += take;
        }
      }
      if (nsel == 0) break;
      if (c_exp >= a.max_exp) { status = PEOS_E_OVERFLOW; break; }
      hint = (W == 1) ? my_pos : __shfl_sync(kFull, my_pos, 0);
      int32_t my_v = -1;
      float my_d = 0.0f;
      if (W == 1 || lane < nsel) {
        my_v = s_ri[my_pos];
        my_d = s_rd[my_pos];
      }
#ifdef PEOS_CHECKED
      if (__any_sync(kFull, (W == 1 ? lane == 0 : lane < nsel) &&
                                !PEOS_EXPECT(my_v >= 0 && (long long)my_v < a.n, kChkExpanded))) {
        status = PEOS_E_INVAL;
        break;
      }
#endif
      __syncwarp();
      if (W == 1 ? lane == 0 : lane < nsel) s_ri[my_pos] = my_v | kExpanded;
      c_exp += nsel;
      const bool full = (len == ef);
      const float delta2 = full ? s_rd[ef - 1] : INFINITY;
      const bool testing = ROUTING && full && a.K.mode != 2;
      c_full += full ? nsel : 0;
      if (W > 1 && nsel > 1) {
        // the later nodes' edge data into L2 while the first node is tested
        const size_t span = testing ? a.rec_stride : (size_t)4 * R;
        const int lines = (int)((span + 127) >> 7);
        for (int w = 1; w < nsel; ++w) {
          const int32_t vw = __shfl_sync(kFull, my_v, w);
          const char* p = testing ? reinterpret_cast<const char*>(a.rec + (size_t)vw * a.rec_stride)
                        : ROUTING != 0 ? reinterpret_cast<const char*>(a.rec + (size_t)vw * a.rec_stride +
                                                                        rec_ids_offset(R, kSB))
                                       : reinterpret_cast<const char*>(a.nbrs + (size_t)vw * R);
          for (int l = lane; l < lines; l += 32) prefetch_l2(p + ((size_t)l << 7));
        }
      }

      // ---- edge groups.  With one node per iteration an out-degree up to 64 is taken in
      //      groups of 32 edges, one edge per lane: the second group only when the node
      //      has an edge in slots 32..R-1 (found while the first group loads).  δ and
      //      "|R| = efs" stay those of the iteration's start for both groups, and the
      //      second group's passes are inserted after the first's: the list keeps the efs
      //      smallest of all the candidates either way, as one sorted insertion would.
      const int ngroup = (kGroups && R > 32) ? 2 : 1;
      bool more = false;
      for (int grp = 0; grp < ngroup; ++grp) {
      if (grp == 1 && !more) break;
      const int gb = grp * 32;  // first slot of the group
      do {  // a `continue` below ends this group

      // ---- each selected node in turn: its edge data, the visited filter and the routing
      //      test; passes are appended to the iteration's candidates and marked visited,
      //      so a later node of the iteration skips them
      int npass = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        if (w < nsel) {
          const int32_t v = (W == 1) ? my_v : __shfl_sync(kFull, my_v, w);
          const float dv = (W == 1) ? my_d : __shfl_sync(kFull, my_d, w);
          const float xn = sqrtf(dv);
          const float inv = 1.0f / xn;

          // edge data of v.  Under the test every lane loads its own edge's id, ||e||,
          // w_reg, sqrt(L) w_res, node term and packed codes straight into registers: one
          // round trip.
          int32_t id[NL];
          float en[NL], wr[NL], cr[NL], sv[NL];
          unsigned long long cw[NL][CW];
          if (testing) {
            const uint8_t* rv = a.rec + (size_t)v * a.rec_stride;
            const int32_t* ri = reinterpret_cast<const int32_t*>(rv + rec_ids_offset(R, kSB));
            const unsigned long long* rc = reinterpret_cast<const unsigned long long*>(rv + rec_codes_offset(R, kSB));
            float4 step = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kSB != 32) step = __ldg(reinterpret_cast<const float4*>(rv));  // the node's quantisation steps
#pragma unroll
            for (int r = 0; r < NL; ++r) {
              const int sl = gb + r * 32 + lane;
              id[r] = -1;
              if (sl < R) {
                id[r] = __ldg(ri + sl);
                if constexpr (kSB == 32) {
                  const float4 f = __ldg(reinterpret_cast<const float4*>(rv) + sl);
                  en[r] = f.x;
                  wr[r] = f.y;
                  cr[r] = f.z;
                  sv[r] = f.w;
                } else if constexpr (kSB == 16) {
                  const short4 qv = __ldg(reinterpret_cast<const short4*>(rv + rec_q_offset(R)) + sl);
                  en[r] = (float)qv.x * step.x;
                  wr[r] = (float)qv.y * step.y;
                  cr[r] = (float)qv.z * step.z;
                  sv[r] = __ldg(reinterpret_cast<const float*>(rv + rec_sv_offset(R)) + sl);
                } else {  // {char4 q, float sv} in one 8-byte load
                  const uint2 pr = __ldg(reinterpret_cast<const uint2*>(rv + rec_pair_offset()) + sl);
                  en[r] = (float)(int8_t)(pr.x & 0xffu) * step.x;
                  wr[r] = (float)(int8_t)((pr.x >> 8) & 0xffu) * step.y;
                  cr[r] = (float)(int8_t)((pr.x >> 16) & 0xffu) * step.z;
                  sv[r] = __uint_as_float(pr.y);
                }
#pragma unroll
                for (int cwi = 0; cwi < CW; ++cwi)
                  cw[r][cwi] = (cwi < a.code_words) ? __ldg(rc + (size_t)cwi * R + sl) : 0ull;
              }
            }
          } else {
#pragma unroll
            for (int r = 0; r < NL; ++r) {
              const int sl = gb + r * 32 + lane;
              id[r] = -1;
              if (sl < R)
                id[r] = ROUTING != 0 ? __ldg(reinterpret_cast<const int32_t*>(a.rec + (size_t)v * a.rec_stride +
                                                                         rec_ids_offset(R, kSB)) + sl)
                                : __ldg(a.nbrs + (size_t)v * R + sl);
            }
          }
          if (kGroups && R > 32 && grp == 0) {
            // does the node have an edge in the second group?  The index's per-node flag
            // (one byte, in the same round trip), else the group's ids themselves
            if (a.wide) {
              more = __ldg(a.wide + v) != 0;
            } else {
              int32_t id2 = -1;
              if (32 + lane < R)
                id2 = ROUTING != 0 ? __ldg(reinterpret_cast<const int32_t*>(a.rec + (size_t)v * a.rec_stride +
                                                                       rec_ids_offset(R, kSB)) + 32 + lane)
                                   : __ldg(a.nbrs + (size_t)v * R + 32 + lane);
              more = __any_sync(kFull, id2 >= 0);
            }
          }

          // frame Q: v.q and r = ||p||^2/2 - p.q from the distances and squared norms
          // (||q - o||^2 = ||q||^2 + ||o||^2 - 2 q.o), p the efs-th entry of R
          float vq = 0.0f, rq = 0.0f;
          if (kFrameQ && testing) {
            const float vv = __ldg(a.norms + v);
            const float pp = __ldg(a.norms + (s_ri[ef - 1] & ~kExpanded));
            vq = ((qq + vv) - dv) / 2.0f;
            rq = pp / 2.0f - ((qq + pp) - delta2) / 2.0f;
          }

          // SimHash: the bits of x = q - v, [S_i . q - S_i . v >= 0], one ballot per 32 bits
          unsigned long long bx[CW];
          if (ROUTING == 2) {
#pragma unroll
            for (int cwi = 0; cwi < CW; ++cwi) {
              bx[cwi] = 0ull;
              if (testing && cwi < a.code_words) {
                const float* tvv = a.sh_tv + (size_t)v * a.sh_K + 64 * cwi;
                const unsigned lo = __ballot_sync(kFull, s_tq[64 * cwi + lane] - __ldg(tvv + lane) >= 0.0f);
                const unsigned hi = __ballot_sync(kFull, s_tq[64 * cwi + 32 + lane] - __ldg(tvv + 32 + lane) >= 0.0f);
                bx[cwi] = (unsigned long long)lo | ((unsigned long long)hi << 32);
              }
            }
          }

          // ---- visited filter and routing test
          bool pass[NL];
          unsigned pm[NL];
#pragma unroll
          for (int r = 0; r < NL; ++r) {
            if ((long long)id[r] >= a.n) id[r] = -1;  // never read outside the base
            bool cand = id[r] >= 0;
            if (COUNT) c_edges += cand ? 1 : 0;
            if (cand && visit_seen(s_vis, id[r], hb)) {
              cand = false;
              if (COUNT) ++c_vskip;
            }
            bool p = cand;
            if (testing && cand) {
              float Ao, Ho, To;
              const int kind =
                  ROUTING == 2 ? simhash_edge_test(s_acrit, a.sh_K, a.code_words, bx, cw[r], dv, xn, delta2, en[r],
                                                   a.K.mode, p)
                  : kFrameQ ? peos_edge_test_q(s_tq, vq, rq, __ldg(a.norms + id[r]), qn, cw[r], a.code_bits,
                                                    a.codes_per_word, en[r], wr[r], cr[r], a.K, p)
                                 : peos_edge_test<false>(s_tq, sv[r], dv, xn, inv, delta2, cw[r], a.code_bits,
                                                         a.codes_per_word, en[r], wr[r], cr[r], a.K, p, Ao, Ho, To);
              if (COUNT) {
                c_arej += kind == kRejectA;
                c_aacc += kind == kAcceptA;
                if (kind == kDecidedH) {
                  ++c_htest;
                  c_hpass += p ? 1 : 0;
                }
              }
            }
            if (NRC == 1) {
              // a node listed twice in one row passes once (the first slot), as a visited
              // set updated in slot order would have it; wider candidate sets drop repeats
              // at the merge instead
              const unsigned peers = __match_any_sync(kFull, id[r]);
              const unsigned pmask = __ballot_sync(kFull, p);
              if (p && (peers & pmask & ((1u << lane) - 1u))) p = false;
            }
            pass[r] = p;
            pm[r] = __ballot_sync(kFull, p);
          }
          {
            int before = npass;
#pragma unroll
            for (int r = 0; r < NL; ++r) {
              if (pass[r]) {
                const int slot = before + __popc(pm[r] & ((1u << lane) - 1u));
                visit_mark(s_vis, id[r], hb);
                if (PEOS_EXPECT(slot < kCand && id[r] >= 0 && (long long)id[r] < a.n, kChkCandidate)) s_cid[slot] = id[r];
              }
              before += __popc(pm[r]);
            }
            npass = before;
          }
          __syncwarp();
        }
      }
      if (npass == 0) continue;

      // ---- exact distances of the passing neighbours: rows past the first batch
      //      are prefetched into L2 so that every batch after the first hits L2; rows
      //      longer than 8 lines (each lane loads several chunks of a row, one after the
      //      other) are all prefetched, the first batch too, so that its chunks arrive
      //      together
      if (pf_row < pf_rows) {
        const int pf_first = lines_per_row > 8 ? 0 : kGather;
        for (int rr = pf_first + pf_row; rr < npass; rr += pf_rows) {
          const char* row = reinterpret_cast<const char*>(a.X) + (size_t)s_cid[rr] * row_bytes;
          for (int l = pf_line; l < lines_per_row; l += 32) prefetch_l2(row + ((size_t)l << 7));
        }
      }
      float mydist[NRC];
#pragma unroll
      for (int r = 0; r < NRC; ++r) mydist[r] = INFINITY;
      for (int b = 0; b < npass; b += kGather)
        gather_batch<kGather, NRC, DT>(q4, a.X, a.scales, d4, s_cid, b, min(kGather, npass - b), lane, mydist);
      c_ndist += npass;

      // ---- candidates that can enter R: below the list bound (or the list is not full)
      //      and not already in R (a node forgotten by the visited table); for each,
      //      its insertion position in R by binary search on (dist, id)
      uint64_t key[NRC];
      int pos[NRC];
      unsigned km[NRC];  // kept candidates of each register: bit `lane` = this lane's
      int nkeep = 0;
#pragma unroll
      for (int r = 0; r < NRC; ++r) {
        const int g = r * 32 + lane;
        key[r] = kNoKey;
        pos[r] = 0;
        bool keep = false;
        if (g < npass && (!full || mydist[r] < delta2)) {
          const float kd = mydist[r];
          const int32_t kid = s_cid[g];
          key[r] = pack_key(kd, kid);
          int lo = 0, hi = len;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const float md = s_rd[mid];
            const int32_t mi = s_ri[mid] & ~kExpanded;
            const bool less = (md < kd) || (md == kd && mi < kid);
            if (less) lo = mid + 1; else hi = mid;
          }
          pos[r] = lo;
          keep = !(lo < len && s_rd[lo] == kd && (s_ri[lo] & ~kExpanded) == kid);
        }
        km[r] = __ballot_sync(kFull, keep);
        nkeep += __popc(km[r]);
      }
      if (nkeep == 0) continue;

      int J;
      if constexpr (NRC == 1) {
        // ---- rank of each kept candidate among the kept ones (ascending (dist, id))
        int rank = 0;
        {
          unsigned m = km[0];
          while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint64_t other = __shfl_sync(kFull, key[0], src);
            rank += (other < key[0]) ? 1 : 0;
          }
        }
        // ---- Algorithm 1's rule in sorted order: the candidate of rank g enters iff every
        //      candidate before it did and dist < the (ef-1-g)-th entry of R (entries past
        //      len count as +inf); J = number entering
        const bool keep0 = (km[0] >> lane) & 1u;
        int fail_rank = 0x7fffffff;
        if (keep0) {
          const int idx = ef - 1 - rank;
          const float bound = idx < 0 ? -INFINITY : (idx < len ? s_rd[idx] : INFINITY);
          if (!(key_dist(key[0]) < bound)) fail_rank = rank;
        }
        J = min(nkeep, __reduce_min_sync(kFull, fail_rank));
        if (J == 0) continue;
        if (keep0 && rank < J) {
          s_ckey[rank] = key[0];
          s_cpos[rank] = pos[0];
        }
        __syncwarp();
      } else {
        // ---- rank of each kept candidate, ties (the same node passed twice in this
        //      iteration) broken by candidate index, so every kept candidate has its own
        //      slot in ascending (dist, id)
        int rank[NRC];
#pragma unroll
        for (int r = 0; r < NRC; ++r) rank[r] = 0;
#pragma unroll
        for (int rs = 0; rs < NRC; ++rs) {
          unsigned m = km[rs];
          while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint64_t other = __shfl_sync(kFull, key[rs], src);
            const int oi = rs * 32 + src;
#pragma unroll
            for (int r = 0; r < NRC; ++r)
              rank[r] += ((other < key[r]) || (other == key[r] && oi < r * 32 + lane)) ? 1 : 0;
          }
        }
#pragma unroll
        for (int r = 0; r < NRC; ++r) {
          if (((km[r] >> lane) & 1u) && PEOS_EXPECT(rank[r] < kCand, kChkListWrite)) {
            s_ckey[rank[r]] = key[r];
            s_cpos[rank[r]] = pos[r];
          }
        }
        __syncwarp();
        // ---- drop repeats (equal keys are adjacent), compacting in place: an entry moves
        //      only to a lower slot, and every slot is read before it is written
        int nk = 0;
        for (int b = 0; b < nkeep; b += 32) {
          const int g = b + lane;
          uint64_t kk = kNoKey;
          int pp = 0;
          bool first = false;
          if (g < nkeep) {
            kk = s_ckey[g];
            pp = s_cpos[g];
            first = (g == 0) || (s_ckey[g - 1] != kk);
          }
          const unsigned bal = __ballot_sync(kFull, first);
          __syncwarp();
          if (first) {
            const int dst = nk + __popc(bal & ((1u << lane) - 1u));
            s_ckey[dst] = kk;
            s_cpos[dst] = pp;
          }
          nk += __popc(bal);
          __syncwarp();
        }
        // ---- Algorithm 1's rule in sorted order (as above) over the distinct candidates
        J = nk;
        for (int b = 0; b < nk; b += 32) {
          const int g = b + lane;
          int fail = 0x7fffffff;
          if (g < nk) {
            const int idx = ef - 1 - g;
            const float bound = idx < 0 ? -INFINITY : (idx < len ? s_rd[idx] : INFINITY);
            if (!(key_dist(s_ckey[g]) < bound)) fail = g;
          }
          J = min(J, __reduce_min_sync(kFull, fail));
        }
        if (J == 0) continue;
      }

      // ---- in-place merge: shift R's tail from the back, then write the new entries
      const int p0 = s_cpos[0];
      for (int top = len - 1; top >= p0; top -= 32) {
        const int i = top - lane;
        float dd = 0.0f;
        int32_t ii = 0;
        int ni = ef;
        if (i >= p0) {
          dd = s_rd[i];
          ii = s_ri[i];
          int lo = 0, hi = J;  // number of accepted candidates with cpos <= i
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_cpos[mid] <= i) lo = mid + 1; else hi = mid;
          }
          ni = i + lo;
        }
        __syncwarp();
        if (i >= p0 && ni < ef && PEOS_EXPECT(ni > i, kChkListWrite)) {
          s_rd[ni] = dd;
          s_ri[ni] = ii;
        }
        __syncwarp();
      }
      for (int g = lane; g < J; g += 32) {
        const int idx = s_cpos[g] + g;
        const uint64_t kk = s_ckey[g];
        if (PEOS_EXPECT(idx >= 0 && idx < ef, kChkListWrite)) {
          s_rd[idx] = key_dist(kk);
          s_ri[idx] = key_id(kk);
        }
      }
      len = min(ef, len + J);
#ifdef PEOS_CHECKED
      __syncwarp();
      check_list(s_rd, s_ri, len, lane, a.check);
#endif
      hint = min(hint, p0);
      c_ins += J;
      __syncwarp();
      } while (0);
      }
    }

    // ---- outputs
    for (int j = lane; j < a.k; j += 32) {
      const bool have = j < len && j < kq;
      a.ids_out[(size_t)qi * a.k + j] = have ? (s_ri[j] & ~kExpanded) : -1;
      a.dists_out[(size_t)qi * a.k + j] = have ? s_rd[j] : INFINITY;
    }
    if (COUNT) {
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

template <int ROUTING, int NR, int DT, int G, int W, int CW, bool QG = false>
int resident_ctas(const KArgs& ka, int warps, size_t smem_total) {
  auto fn = ka.counters ? search_kernel<ROUTING, NR, true, DT, G, W, CW, QG>
                        : search_kernel<ROUTING, NR, false, DT, G, W, CW, QG>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_total) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem_total) != cudaSuccess) return 0;
  return per_sm;
}

template <int ROUTING, int NR, int DT, int G, int W, int CW, bool QG = false>
cudaError_t launch_t(const KArgs& ka, int warps, size_t smem_total, cudaStream_t st) {
  auto fn = ka.counters ? search_kernel<ROUTING, NR, true, DT, G, W, CW, QG>
                        : search_kernel<ROUTING, NR, false, DT, G, W, CW, QG>;
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

// One kernel variant for the graph's out-degree: R <= 32 one edge per lane; up to 64 the
// NR = 2 form (a routing test with one node per iteration: one edge per lane in two groups
// of 32; plain routing or a beam width W > 1: two edges per lane).
template <int ROUTING, int DT, int G, int W, int CW, bool QG = false>
cudaError_t launch_r(const KArgs& ka, int R, int warps, size_t smem_total, cudaStream_t st) {
  return R <= 32 ? launch_t<ROUTING, 1, DT, G, W, CW, QG>(ka, warps, smem_total, st)
                 : launch_t<ROUTING, 2, DT, G, W, CW, QG>(ka, warps, smem_total, st);
}
template <int ROUTING, int DT, int G, int W, int CW, bool QG = false>
int resident_r(const KArgs& ka, int R, int warps, size_t smem_total) {
  return R <= 32 ? resident_ctas<ROUTING, 1, DT, G, W, CW, QG>(ka, warps, smem_total)
                 : resident_ctas<ROUTING, 2, DT, G, W, CW, QG>(ka, warps, smem_total);
}

// Launch the search over a stored base of element type DT with CW code words per edge
// (each (DT, CW) explicitly instantiated in its own translation unit), one node per
// iteration.  Plain routing reads no codes: it is built for CW = 1 only.
template <int DT, int G, int CW>
cudaError_t launch_search_shaped(const KArgs& ka, int routing, int R, int warps, size_t smem_total,
                                 cudaStream_t st) {
  // routing = the kernel variant (see search_kernel); the SimHash baseline and frame Q
  // read FP32 rows only; plain routing and PEOs in frame T (plain, permuted or compact
  // records) read every stored type
  if (routing == 0 && CW != 1) return cudaErrorInvalidValue;
  if (ka.d >= 512 && (routing == 0 || routing == 1)) {
    // long rows: the query may stay in global memory (read through L1 beside the rows),
    // which is worth it when its shared-memory copy is what limits the resident CTAs
    const size_t qb = align16((size_t)ka.d * 4);
    KArgs kq = ka;
    for (int i = 0; i < kNumOff; ++i)
      if (i != kOffQ) kq.off[i] -= (int)qb;  // the query's slice comes first in the layout
    kq.smem_per_warp -= (int)qb;
    const size_t total_q = smem_total - (size_t)warps * qb;
    if (routing == 0) {
      if constexpr (CW == 1) {
        if (resident_r<0, DT, G, 1, CW, true>(kq, R, warps, total_q) > resident_r<0, DT, G, 1, CW>(ka, R, warps, smem_total))
          return launch_r<0, DT, G, 1, CW, true>(kq, R, warps, total_q, st);
      }
    } else {
      if (resident_r<1, DT, G, 1, CW, true>(kq, R, warps, total_q) > resident_r<1, DT, G, 1, CW>(ka, R, warps, smem_total))
        return launch_r<1, DT, G, 1, CW, true>(kq, R, warps, total_q, st);
    }
  }
  switch (routing) {
    case 0:
      if constexpr (CW == 1) return launch_r<0, DT, G, 1, CW>(ka, R, warps, smem_total, st);
      break;
    case 1: return launch_r<1, DT, G, 1, CW>(ka, R, warps, smem_total, st);
    case 4: return launch_r<4, DT, G, 1, CW>(ka, R, warps, smem_total, st);
    case 6: return launch_r<6, DT, G, 1, CW>(ka, R, warps, smem_total, st);
    case 7: return launch_r<7, DT, G, 1, CW>(ka, R, warps, smem_total, st);
    default: break;
  }
  if constexpr (DT == kF32) {
    switch (routing) {
      case 2: return launch_r<2, DT, G, 1, CW>(ka, R, warps, smem_total, st);
      case 3: return launch_r<3, DT, G, 1, CW>(ka, R, warps, smem_total, st);
      case 5: return launch_r<5, DT, G, 1, CW>(ka, R, warps, smem_total, st);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

// gather = rows per gather batch (4 or 8; 0 = the routing method's default)
template <int DT, int CW>
cudaError_t launch_search_typed(const KArgs& ka, int routing, int R, int gather, int warps, size_t smem_total,
                                cudaStream_t st) {
  if (gather == 0) gather = default_gather(routing);
  if (gather == 8) return launch_search_shaped<DT, 8, CW>(ka, routing, R, warps, smem_total, st);
  if (gather == 4) return launch_search_shaped<DT, 4, CW>(ka, routing, R, warps, smem_total, st);
  return cudaErrorInvalidValue;
}

// Beam width W = 2 or 4 (nodes expanded per iteration): plain routing and PEOs in frame T
// (kernel variants 0 and 1), every stored type.
template <int DT, int W, int CW>
cudaError_t launch_search_beam_w(const KArgs& ka, int routing, int R, int gather, int warps, size_t smem_total,
                                 cudaStream_t st) {
  if (gather == 0) gather = default_gather(routing);
  if (gather != 4 && gather != 8) return cudaErrorInvalidValue;
  if (routing == 0) {
    if constexpr (CW == 1) {
      if (gather == 8) return launch_r<0, DT, 8, W, CW>(ka, R, warps, smem_total, st);
      return launch_r<0, DT, 4, W, CW>(ka, R, warps, smem_total, st);
    }
    return cudaErrorInvalidValue;
  }
  if (routing == 1) {
    if (gather == 8) return launch_r<1, DT, 8, W, CW>(ka, R, warps, smem_total, st);
    return launch_r<1, DT, 4, W, CW>(ka, R, warps, smem_total, st);
  }
  return cudaErrorInvalidValue;
}

template <int DT, int CW>
cudaError_t launch_search_beam(const KArgs& ka, int routing, int R, int gather, int beam, int warps,
                               size_t smem_total, cudaStream_t st) {
  if (beam == 2) return launch_search_beam_w<DT, 2, CW>(ka, routing, R, gather, warps, smem_total, st);
  if (beam == 4) return launch_search_beam_w<DT, 4, CW>(ka, routing, R, gather, warps, smem_total, st);
  return cudaErrorInvalidValue;
}

#define PEOS_SEARCH_EXTERN(DT, CW)                                                                          \
  extern template cudaError_t launch_search_typed<DT, CW>(const KArgs&, int, int, int, int, size_t, cudaStream_t); \
  extern template cudaError_t launch_search_beam<DT, CW>(const KArgs&, int, int, int, int, int, size_t, cudaStream_t);
PEOS_SEARCH_EXTERN(kF32, 1)
PEOS_SEARCH_EXTERN(kF32, kMaxCodeWords)
PEOS_SEARCH_EXTERN(kBF16, 1)
PEOS_SEARCH_EXTERN(kBF16, kMaxCodeWords)
PEOS_SEARCH_EXTERN(kE4M3, 1)
PEOS_SEARCH_EXTERN(kE4M3, kMaxCodeWords)
#undef PEOS_SEARCH_EXTERN

}  // namespace sk
}  // namespace peos
