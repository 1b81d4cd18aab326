// Exact K-NN by brute force (the recall ground truth): squared l2 distances as
// exact FP32 sums of squared differences, ties broken by id.
//
// Pass 1: a CTA takes 32 queries x one chunk of the base, streams the chunk in
// tiles of 64 points x 128 dims through shared memory (points transposed so a
// lane reads consecutive banks), each warp owning 4 queries; every warp keeps
// its queries' k best (dist, id) keys of the chunk sorted in shared memory and
// writes them to scratch [nq][chunks][k].
// Pass 2: one warp per query merges its chunks' lists into the final k.
#include <cuda_runtime.h>
#include <math.h>

#include "device.cuh"
#include "internal.h"

namespace peos {
namespace {

constexpr int kQT = 32;      // queries per CTA
constexpr int kPT = 64;      // points per tile
constexpr int kDK = 128;     // dims per slab
constexpr int kChunk = 16384;
constexpr int kThreads = 256;

// Insert `key` into the sorted list `lst` of length k if it beats the last entry.
// Called by a whole warp with the same key.
__device__ __forceinline__ void warp_list_insert(uint64_t* lst, int k, uint64_t key, int lane) {
  if (!(key < lst[k - 1])) return;
  // position = number of entries < key
  int cnt = 0;
  for (int b = 0; b < k; b += 32) {
    const int i = b + lane;
    const bool lt = (i < k) && (lst[i] < key);
    cnt += __popc(__ballot_sync(kFull, lt));
  }
  // shift [cnt, k-1) right by one, from the back in chunks
  for (int top = k - 2; top >= cnt; top -= 32) {
    const int i = top - lane;
    uint64_t val = 0;
    if (i >= cnt) val = lst[i];
    __syncwarp();
    if (i >= cnt) lst[i + 1] = val;
    __syncwarp();
  }
  if (lane == 0) lst[cnt] = key;
  __syncwarp();
}

__global__ void __launch_bounds__(kThreads) knn_chunk_kernel(const float* __restrict__ X, long long n, int d,
                                                             const float* __restrict__ Q, long long nq, int k,
                                                             int nchunks, uint64_t* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* qs = reinterpret_cast<float*>(smem_raw);          // [kQT][kDK]
  float* xs = qs + kQT * kDK;                               // [kDK][kPT]
  uint64_t* lists = reinterpret_cast<uint64_t*>(xs + kDK * kPT);  // [kQT][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long q0 = (long long)blockIdx.x * kQT;
  const int chunk = blockIdx.y;
  const long long p_begin = (long long)chunk * kChunk;
  const long long p_end = min(n, p_begin + kChunk);

  for (int i = tid; i < kQT * k; i += kThreads) lists[i] = kNoKey;
  __syncthreads();

  for (long long pt = p_begin; pt < p_end; pt += kPT) {
    float acc[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = 0.0f;
    for (int k0 = 0; k0 < d; k0 += kDK) {
      const int dk = min(kDK, d - k0);
      // stage queries [kQT][dk] and points transposed [dk][kPT]
      for (int i = tid; i < kQT * (kDK / 4); i += kThreads) {
        const int qq = i / (kDK / 4), c4 = i - qq * (kDK / 4);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q0 + qq < nq && c4 * 4 < dk) v = *reinterpret_cast<const float4*>(Q + (size_t)(q0 + qq) * d + k0 + c4 * 4);
        *reinterpret_cast<float4*>(qs + qq * kDK + c4 * 4) = v;
      }
      for (int i = tid; i < kPT * (kDK / 4); i += kThreads) {
        const int p = i % kPT, c4 = i / kPT;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pt + p < p_end && c4 * 4 < dk) v = __ldg(reinterpret_cast<const float4*>(X + (size_t)(pt + p) * d + k0 + c4 * 4));
        xs[(c4 * 4 + 0) * kPT + p] = v.x;
        xs[(c4 * 4 + 1) * kPT + p] = v.y;
        xs[(c4 * 4 + 2) * kPT + p] = v.z;
        xs[(c4 * 4 + 3) * kPT + p] = v.w;
      }
      __syncthreads();
      const float* qw = qs + (warp * 4) * kDK;
      for (int kk = 0; kk < dk; ++kk) {
        const float x0 = xs[kk * kPT + lane], x1 = xs[kk * kPT + lane + 32];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float qv = qw[a * kDK + kk];
          const float t0 = qv - x0, t1 = qv - x1;
          acc[a][0] = fmaf(t0, t0, acc[a][0]);
          acc[a][1] = fmaf(t1, t1, acc[a][1]);
        }
      }
      __syncthreads();
    }
    // top-k update for the warp's 4 queries
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      uint64_t* lst = lists + (warp * 4 + a) * k;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long p = pt + lane + 32 * h;
        uint64_t key = kNoKey;
        if (p < p_end) key = pack_key(acc[a][h], (int32_t)p);
        unsigned want = __ballot_sync(kFull, key < lst[k - 1]);
        while (want) {
          const int src = __ffs(want) - 1;
          want &= want - 1;
          const uint64_t kk = __shfl_sync(kFull, key, src);
          warp_list_insert(lst, k, kk, lane);
        }
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < kQT * k; i += kThreads) {
    const int qq = i / k, j = i - qq * k;
    if (q0 + qq < nq) part[((size_t)(q0 + qq) * nchunks + chunk) * k + j] = lists[i];
  }
}

__global__ void knn_merge_kernel(const uint64_t* __restrict__ part, long long nq, int k, int nchunks,
                                 int32_t* __restrict__ ids_out, float* __restrict__ dists_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  uint64_t* lst = reinterpret_cast<uint64_t*>(smem_raw) + (size_t)warp * k;
  for (long long q = (long long)blockIdx.x * wpb + warp; q < nq; q += (long long)gridDim.x * wpb) {
    for (int i = lane; i < k; i += 32) lst[i] = kNoKey;
    __syncwarp();
    const uint64_t* src = part + (size_t)q * nchunks * k;
    const int total = nchunks * k;
    for (int b = 0; b < total; b += 32) {
      const int i = b + lane;
      const uint64_t key = i < total ? src[i] : kNoKey;
      unsigned want = __ballot_sync(kFull, key < lst[k - 1]);
      while (want) {
        const int s = __ffs(want) - 1;
        want &= want - 1;
        const uint64_t kk = __shfl_sync(kFull, key, s);
        warp_list_insert(lst, k, kk, lane);
      }
    }
    for (int i = lane; i < k; i += 32) {
      const uint64_t key = lst[i];
      ids_out[(size_t)q * k + i] = key == kNoKey ? -1 : key_id(key);
      dists_out[(size_t)q * k + i] = key == kNoKey ? INFINITY : key_dist(key);
    }
    __syncwarp();
  }
}

}  // namespace

size_t knn_scratch_bytes(int64_t n, int64_t nq, int k) {
  const int64_t nchunks = (n + kChunk - 1) / kChunk;
  return (size_t)nq * (size_t)nchunks * (size_t)k * sizeof(uint64_t);
}

cudaError_t launch_knn(const float* X, int64_t n, int d, const float* Q, int64_t nq, int k, int32_t* ids_out,
                       float* dists_out, void* scratch, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  const int nchunks = (int)((n + kChunk - 1) / kChunk);
  uint64_t* part = static_cast<uint64_t*>(scratch);
  const size_t smem1 = sizeof(float) * (kQT * kDK + kDK * kPT) + sizeof(uint64_t) * (size_t)kQT * k;
  cudaError_t e = cudaFuncSetAttribute(knn_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
  if (e != cudaSuccess) return e;
  dim3 grid1((unsigned)((nq + kQT - 1) / kQT), (unsigned)nchunks);
  knn_chunk_kernel<<<grid1, kThreads, smem1, st>>>(X, n, d, Q, nq, k, nchunks, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int wpb = 4;
  const size_t smem2 = sizeof(uint64_t) * (size_t)wpb * k;
  e = cudaFuncSetAttribute(knn_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  if (e != cudaSuccess) return e;
  long long g2 = (nq + wpb - 1) / wpb;
  if (g2 > 65535) g2 = 65535;
  knn_merge_kernel<<<(unsigned)g2, wpb * 32, smem2, st>>>(part, nq, k, nchunks, ids_out, dists_out);
  return cudaGetLastError();
}

}  // namespace peos
