// Hierarchical entry (the paper's HNSW indexes, Sec. 6.1): each query descends from the
// top layer's entry through the upper layers by greedy search with a list of one, and
// the node it ends on in the lowest upper layer is its entry node for Algorithm 1 on the
// base graph.
//
// One warp per query, persistent CTAs pulling queries from a work counter; the query
// sits in the warp's slice of shared memory.  At the current node c the lanes take its
// out-edges (R_l <= 32, one per lane), the exact distances of the valid ones are gathered
// eight rows at a time by the search's own warp reduction (gather_dists), and a warp
// argmin over (dist, base id) picks the best neighbour; the walk moves there when it is
// strictly closer than c and stops otherwise.  A layer's node moves to the layer below
// through the layer's `down` map.  Every walk is bounded by the layer's node count (the
// distance strictly decreases, so that bound is never reached by a valid layer).
#include <cuda_runtime.h>

#include "search_kernel.cuh"

namespace peos {
namespace {

using namespace sk;

constexpr int kHierWarps = 8;

struct Layers {
  int levels;
  int top_entry;
  long long n[kMaxHierLevels];
  int R[kMaxHierLevels];
  const int32_t* ids[kMaxHierLevels];
  const int32_t* nbrs[kMaxHierLevels];
  const int32_t* down[kMaxHierLevels];
};

template <int DT>
__global__ void __launch_bounds__(kHierWarps * 32, 4) hier_entry_kernel(Layers L, const void* __restrict__ X,
                                                                    const float* __restrict__ scales,
                                                                    long long nbase, int d,
                                                                    const float* __restrict__ Q, long long nq,
                                                                    int* __restrict__ work,
                                                                    int32_t* __restrict__ entries) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* s_q = reinterpret_cast<float*>(smem_raw) + (size_t)warp * d;
  const float4* q4 = reinterpret_cast<const float4*>(s_q);
  const int d4 = d >> 2;
  for (;;) {
    int slot = 0;
    if (lane == 0) slot = atomicAdd(work, 1);
    slot = __shfl_sync(kFull, slot, 0);
    if ((long long)slot >= nq) break;
    const float4* qg = reinterpret_cast<const float4*>(Q + (size_t)slot * d);
    __syncwarp();
    for (int c = lane; c < d4; c += 32) reinterpret_cast<float4*>(s_q)[c] = __ldg(qg + c);
    __syncwarp();
    // ids that leave their layer or the base end the walk with entry -1 (the search then
    // returns an empty row with PEOS_E_INVAL for the query)
    int cur = L.top_entry;  // local id in the current layer (checked on the host)
    int32_t gid[8];
    gid[0] = __ldg(L.ids[0] + cur);
    bool ok = gid[0] >= 0 && (long long)gid[0] < nbase;
    float dc = 0.0f;
    if (ok) dc = __shfl_sync(kFull, gather_dists<8, DT>(q4, X, scales, d4, gid, 1, lane), row_lane<8>(0));
    for (int l = 0; ok && l < L.levels; ++l) {
      const int32_t* ids = L.ids[l];
      const int32_t* nbrs = L.nbrs[l];
      const int R = L.R[l];
      const long long nl = L.n[l];
      for (long long hop = 0; hop < nl; ++hop) {
        int u = lane < R ? __ldg(nbrs + (size_t)cur * R + lane) : -1;
        if ((long long)u >= nl) u = -1;
        int32_t g = u >= 0 ? __ldg(ids + u) : -1;
        if (g < 0 || (long long)g >= nbase) {
          u = -1;
          g = -1;
        }
        unsigned valid = __ballot_sync(kFull, u >= 0);
        float du = INFINITY;
        // gather the valid neighbours' distances, 8 rows per batch, in lane order
        while (valid) {
          int lanes[8];
          int cnt = 0;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            lanes[j] = valid ? __ffs(valid) - 1 : 0;
            if (valid) {
              valid &= valid - 1;
              ++cnt;
            }
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) gid[j] = __shfl_sync(kFull, g, lanes[j]);
          const float tot = gather_dists<8, DT>(q4, X, scales, d4, gid, cnt, lane);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float v = __shfl_sync(kFull, tot, row_lane<8>(j));
            if (j < cnt && lane == lanes[j]) du = v;
          }
        }
        // warp argmin over (dist, base id)
        float bd = du;
        int32_t bg = g, bu = u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float od = __shfl_xor_sync(kFull, bd, o);
          const int32_t og = __shfl_xor_sync(kFull, bg, o);
          const int32_t ou = __shfl_xor_sync(kFull, bu, o);
          const bool take = ou >= 0 && (bu < 0 || od < bd || (od == bd && og < bg));
          if (take) {
            bd = od;
            bg = og;
            bu = ou;
          }
        }
        if (bu < 0 || !(bd < dc)) break;
        cur = bu;
        dc = bd;
      }
      if (l + 1 < L.levels) {
        cur = __ldg(L.down[l] + cur);
        ok = cur >= 0 && (long long)cur < L.n[l + 1];
      }
    }
    int32_t out = ok ? __ldg(L.ids[L.levels - 1] + cur) : -1;
    if (out < 0 || (long long)out >= nbase) out = -1;
    if (lane == 0) entries[slot] = out;
  }
}

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

template <int DT>
cudaError_t launch_typed(const Layers& L, const void* X, const float* scales, long long nbase, int d, const float* Q,
                         long long nq, int* work, int32_t* entries, cudaStream_t st) {
  const size_t smem = (size_t)kHierWarps * d * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(hier_entry_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hier_entry_kernel<DT>, kHierWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)device_sm_count() * per_sm;
  const long long need = (nq + kHierWarps - 1) / kHierWarps;
  if (grid > need) grid = need;
  hier_entry_kernel<DT><<<(unsigned)grid, kHierWarps * 32, smem, st>>>(L, X, scales, nbase, d, Q, nq, work, entries);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_hier_entry(const HierLaunch& h, const void* X, const float* scales, int dtype, int64_t nbase,
                              int d, const float* Q, int64_t nq, int* work, int32_t* entries, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  Layers L;
  L.levels = h.levels;
  L.top_entry = h.top_entry;
  for (int l = 0; l < kMaxHierLevels; ++l) {
    const bool on = l < h.levels;
    L.n[l] = on ? h.n[l] : 0;
    L.R[l] = on ? h.R[l] : 0;
    L.ids[l] = on ? h.ids[l] : nullptr;
    L.nbrs[l] = on ? h.nbrs[l] : nullptr;
    L.down[l] = on ? h.down[l] : nullptr;
  }
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  switch (dtype) {
    case kF32: return launch_typed<kF32>(L, X, scales, nbase, d, Q, nq, work, entries, st);
    case kBF16: return launch_typed<kBF16>(L, X, scales, nbase, d, Q, nq, work, entries, st);
    case kE4M3: return launch_typed<kE4M3>(L, X, scales, nbase, d, Q, nq, work, entries, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace peos
