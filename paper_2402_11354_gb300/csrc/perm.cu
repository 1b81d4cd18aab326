// Dimension permutation of Appendix D.1: the coordinates are dealt to the L subspaces
// so that each subspace carries a similar share of the edges' energy.
//
//   Avg(e_j) = (sum over the edges e = u - v of e_j^2) / |E|   (FP64)
//   coordinates in ascending (Avg, j); d/L rounds; round l gives its L coordinates, in
//   that order, each to the subspace with the greatest running sum of Avg among the
//   subspaces not yet served in the round (equal sums: the lower subspace);
//   perm[i*d' + t] = the t-th coordinate given to subspace i.
//
// Two launches.  edge_sq_kernel: one warp per node, lanes across the coordinates, each
// warp accumulating e_j^2 of its nodes' edges into its own FP64 row of shared memory;
// the CTA then adds its warps' rows (in warp order) into one partial row per CTA.
// assign_kernel (one CTA): adds the CTA partials in CTA order, divides by |E|, sorts
// (Avg, j) with a bitonic network and runs the greedy rounds on one warp (argmax by
// shuffles).  Every FP64 operation is an explicit round-to-nearest intrinsic (no
// contraction); sums of squared differences of integer-valued rows are exact, so the
// permutation is then independent of the summation order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace peos {
namespace {

constexpr int kSqWarps = 8;
constexpr int kAssignThreads = 1024;
constexpr int kMaxPermDim = 2048;

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

// CTAs of edge_sq_kernel: two per SM (fixed for the device, so the partials and their
// order are too)
int sq_grid() { return 2 * device_sms(); }

__global__ void __launch_bounds__(kSqWarps * 32) edge_sq_kernel(const float* __restrict__ X, long long n, int d,
                                                              const int32_t* __restrict__ nbrs, int R,
                                                              double* __restrict__ partial,
                                                              unsigned long long* __restrict__ edges) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* acc = reinterpret_cast<double*>(smem_raw);  // [kSqWarps][d]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* mine = acc + (size_t)warp * d;
  for (int t = lane; t < d; t += 32) mine[t] = 0.0;
  unsigned long long ne = 0;
  for (long long v = (long long)blockIdx.x * kSqWarps + warp; v < n; v += (long long)gridDim.x * kSqWarps) {
    const float* xv = X + (size_t)v * d;
    for (int s = 0; s < R; ++s) {
      const int32_t u = __ldg(nbrs + (size_t)v * R + s);
      if (u < 0) continue;
      ++ne;
      const float* xu = X + (size_t)u * d;
      for (int t = lane; t < d; t += 32) {
        const double e = __dsub_rn((double)__ldg(xu + t), (double)__ldg(xv + t));
        mine[t] = __dadd_rn(mine[t], __dmul_rn(e, e));
      }
    }
  }
  __shared__ unsigned long long s_ne[kSqWarps];
  if (lane == 0) s_ne[warp] = ne;
  __syncthreads();
  for (int t = threadIdx.x; t < d; t += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kSqWarps; ++w) s = __dadd_rn(s, acc[(size_t)w * d + t]);
    partial[(size_t)blockIdx.x * d + t] = s;
  }
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (int w = 0; w < kSqWarps; ++w) tot += s_ne[w];
    edges[blockIdx.x] = tot;
  }
}

// (Avg, j) order: Avg >= 0, so its IEEE bits order like unsigned integers
__device__ __forceinline__ bool key_less(unsigned long long ka, int ja, unsigned long long kb, int jb) {
  return ka < kb || (ka == kb && ja < jb);
}

__global__ void __launch_bounds__(kAssignThreads) assign_kernel(const double* __restrict__ partial,
                                                                const unsigned long long* __restrict__ edges,
                                                                int parts, int d, int L, int p2,
                                                                int32_t* __restrict__ perm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem_raw);  // [p2]
  double* load = reinterpret_cast<double*>(key + p2);                          // [L] running sums
  int* idx = reinterpret_cast<int*>(load + L);                                  // [p2]
  int* cnt = idx + p2;                                                          // [L]
  int* served = cnt + L;                                                        // [L]
  unsigned long long ne = 0;
  for (int b = 0; b < parts; ++b) ne += edges[b];
  for (int j = threadIdx.x; j < p2; j += blockDim.x) {
    if (j < d) {
      double s = 0.0;
      for (int b = 0; b < parts; ++b) s = __dadd_rn(s, partial[(size_t)b * d + j]);
      const double avg = ne ? __ddiv_rn(s, (double)ne) : 0.0;
      key[j] = (unsigned long long)__double_as_longlong(avg);
      idx[j] = j;
    } else {
      key[j] = ~0ull;  // padding sorts last
      idx[j] = j;
    }
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    load[i] = 0.0;
    cnt[i] = 0;
  }
  __syncthreads();
  // bitonic sort of (key, idx) ascending
  for (int size = 2; size <= p2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (p2 >> 1); t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const bool swap = up ? key_less(key[hi], idx[hi], key[lo], idx[lo])
                             : key_less(key[lo], idx[lo], key[hi], idx[hi]);
        if (swap) {
          const unsigned long long k0 = key[lo];
          key[lo] = key[hi];
          key[hi] = k0;
          const int i0 = idx[lo];
          idx[lo] = idx[hi];
          idx[hi] = i0;
        }
      }
      __syncthreads();
    }
  }
  // greedy rounds on warp 0
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const int dp = d / L;
  for (int l = 0; l < dp; ++l) {
    for (int i = lane; i < L; i += 32) served[i] = 0;
    __syncwarp();
    for (int t = 0; t < L; ++t) {
      const int r = l * L + t;
      // the unserved subspace with the greatest sum, lowest index on ties
      int best = -1;
      double bl = 0.0;
      for (int i = lane; i < L; i += 32) {
        if (served[i]) continue;
        if (best < 0 || load[i] > bl) {
          best = i;
          bl = load[i];
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const int ob = __shfl_xor_sync(0xffffffffu, best, o);
        const double ol = __shfl_xor_sync(0xffffffffu, bl, o);
        if (ob >= 0 && (best < 0 || ol > bl || (ol == bl && ob < best))) {
          best = ob;
          bl = ol;
        }
      }
      if (lane == 0) {
        const double v = __longlong_as_double((long long)key[r]);
        served[best] = 1;
        load[best] = __dadd_rn(load[best], v);
        perm[best * dp + cnt[best]] = idx[r];
        cnt[best] += 1;
      }
      __syncwarp();
    }
  }
}

size_t assign_smem(int d, int L, int p2) {
  return (size_t)p2 * 8 + (size_t)L * 8 + (size_t)p2 * 4 + (size_t)L * 4 * 2;
}

}  // namespace

size_t dim_perm_scratch_bytes(int d) {
  const size_t parts = (size_t)sq_grid();
  return parts * (size_t)d * sizeof(double) + parts * sizeof(unsigned long long);
}

cudaError_t launch_dim_permutation(const float* X, int64_t n, int d, const int32_t* nbrs, int R, int L,
                                   void* scratch, int32_t* perm, cudaStream_t st) {
  if (d < 1 || d > kMaxPermDim || L < 1 || d % L != 0) return cudaErrorInvalidValue;
  const int parts = sq_grid();
  double* partial = static_cast<double*>(scratch);
  unsigned long long* edges = reinterpret_cast<unsigned long long*>(partial + (size_t)parts * d);
  const size_t sq_smem = (size_t)kSqWarps * d * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(edge_sq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sq_smem);
  if (e != cudaSuccess) return e;
  edge_sq_kernel<<<parts, kSqWarps * 32, sq_smem, st>>>(X, n, d, nbrs, R, partial, edges);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int p2 = 1;
  while (p2 < d) p2 <<= 1;
  const size_t a_smem = assign_smem(d, L, p2);
  e = cudaFuncSetAttribute(assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a_smem);
  if (e != cudaSuccess) return e;
  assign_kernel<<<1, kAssignThreads, a_smem, st>>>(partial, edges, parts, d, L, p2, perm);
  return cudaGetLastError();
}

}  // namespace peos
