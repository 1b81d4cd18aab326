// Index-time data of the SimHash routing test (Sec. 3.1, Lemma 4.1, with the residual
// remedy: the test hashes e = u - v instead of u): for every edge the K sign bits
// [S_i . e >= 0] (sgn(0) = +1) and ||e||, for every node its table S_i . v.  One CTA per
// node: the node's edges staged in shared memory, one thread per (edge, bit) dot product
// and per table entry; every sum is a plain sequential FP32 sum (compiled with
// --fmad=false), so the bits, norms and tables are reproducible bit for bit.
//
// Thresholds (host): #Col ~ Binomial(K, 1 - theta / pi) for the angle theta between e and
// x = q - v, and u is closer than delta iff theta <= arccos(A).  Hoeffding's bound
// P(#Col <= K p - t) <= exp(-2 t^2 / K) = eps gives t = sqrt(K ln(1/eps) / 2); the test
// passes iff #Col >= K (1 - arccos(A) / pi) - t, i.e. iff A <= cos(pi (1 - (#Col + t) / K)),
// tabulated per #Col in FP64 and rounded once to FP32 (1 where (#Col + t) / K >= 1).
#include <cuda_runtime.h>
#include <math.h>

#include "device.cuh"
#include "internal.h"

namespace peos {
namespace {

constexpr int kShThreads = 256;

__global__ void __launch_bounds__(kShThreads) simhash_build_kernel(const float* __restrict__ X, long long n, int d,
                                                                  const int32_t* __restrict__ nbrs, int R, int K,
                                                                  const float* __restrict__ S,
                                                                  uint8_t* __restrict__ rec, size_t rec_stride,
                                                                  float* __restrict__ tv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* e = reinterpret_cast<float*>(smem_raw);                      // [R][d]
  int32_t* ids = reinterpret_cast<int32_t*>(e + (size_t)R * d);       // [R]
  unsigned char* bit = reinterpret_cast<unsigned char*>(ids + R);     // [R][K]
  const int tid = threadIdx.x;
  const int W = K / 64;
  for (long long v = blockIdx.x; v < n; v += gridDim.x) {
    const float* xv = X + (size_t)v * d;
    for (int s = tid; s < R; s += blockDim.x) ids[s] = nbrs[(size_t)v * R + s];
    __syncthreads();
    for (int idx = tid; idx < R * d; idx += blockDim.x) {
      const int s = idx / d, k = idx - s * d;
      const int32_t u = ids[s];
      e[idx] = u >= 0 ? X[(size_t)u * d + k] - xv[k] : 0.0f;
    }
    // node table S_i . v
    for (int i = tid; i < K; i += blockDim.x) {
      const float* si = S + (size_t)i * d;
      float acc = 0.0f;
      for (int k = 0; k < d; ++k) acc = acc + __ldg(si + k) * __ldg(xv + k);
      tv[(size_t)v * K + i] = acc;
    }
    __syncthreads();
    for (int t = tid; t < R * K; t += blockDim.x) {
      const int s = t / K, i = t - s * K;
      const float* si = S + (size_t)i * d;
      const float* es = e + (size_t)s * d;
      float acc = 0.0f;
      for (int k = 0; k < d; ++k) acc = acc + __ldg(si + k) * es[k];
      bit[t] = (ids[s] >= 0 && acc >= 0.0f) ? 1 : 0;
    }
    __syncthreads();
    uint8_t* r = rec + (size_t)v * rec_stride;
    for (int s = tid; s < R; s += blockDim.x) {
      float en = 0.0f;
      if (ids[s] >= 0) {
        const float* es = e + (size_t)s * d;
        float acc = 0.0f;
        for (int k = 0; k < d; ++k) acc = acc + es[k] * es[k];
        en = sqrtf(acc);
      }
      reinterpret_cast<float4*>(r)[s] = make_float4(en, 0.0f, 0.0f, 0.0f);
      reinterpret_cast<int32_t*>(r + rec_ids_offset(R))[s] = ids[s];
    }
    uint64_t* words = reinterpret_cast<uint64_t*>(r + rec_codes_offset(R));
    for (int t = tid; t < R * W; t += blockDim.x) {
      const int s = t / W, w = t - s * W;
      uint64_t word = 0;
      for (int b = 0; b < 64; ++b) word |= (uint64_t)bit[(size_t)s * K + 64 * w + b] << b;
      words[(size_t)w * R + s] = word;
    }
    for (size_t b = rec_ids_offset(R) + 4 * (size_t)R + tid; b < rec_codes_offset(R); b += blockDim.x) r[b] = 0;
    const size_t used = rec_codes_offset(R) + 8 * (size_t)W * R;
    for (size_t b = used + tid; b < rec_stride; b += blockDim.x) r[b] = 0;
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_simhash_build(const float* X, int64_t n, int d, const int32_t* nbrs, int R, int K, const float* S,
                                 uint8_t* rec, size_t rec_stride, float* tv, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t smem = sizeof(float) * (size_t)R * d + sizeof(int32_t) * (size_t)R + (size_t)R * K;
  cudaError_t e = cudaFuncSetAttribute(simhash_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, simhash_build_kernel, kShThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = (long long)sms * per_sm;
  if (grid > n) grid = n;
  simhash_build_kernel<<<(unsigned)grid, kShThreads, smem, st>>>(X, n, d, nbrs, R, K, S, rec, rec_stride, tv);
  return cudaGetLastError();
}

void simhash_acrit(int K, double eps, float* acrit) {
  const double pi = 3.14159265358979323846;
  const double t = sqrt((double)K * log(1.0 / eps) / 2.0);
  for (int c = 0; c <= K; ++c) {
    const double r = ((double)c + t) / (double)K;
    acrit[c] = r >= 1.0 ? 1.0f : (float)cos(pi * (1.0 - r));
  }
}

}  // namespace peos
