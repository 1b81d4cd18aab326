// Reduced-precision storage of the base vectors for the precision form of the search.
//  - BF16: each FP32 value rounded to the nearest bfloat16 (ties to even); rows unscaled.
//  - FP8 E4M3: one FP32 scale per row, s = max|x| / 448 (1 for an all-zero row), and the
//    codes of x * (448 / max|x|) rounded to the nearest E4M3 value (ties to even) and
//    saturated to +-448, so that s * value(code) approximates x.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"

namespace peos {
namespace {

constexpr int kQuantWarps = 8;

__global__ void __launch_bounds__(kQuantWarps * 32) quantize_kernel(const float* __restrict__ X, long long n, int d,
                                                                    int dtype, void* __restrict__ out,
                                                                    float* __restrict__ scales) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (long long)blockIdx.x * kQuantWarps + (threadIdx.x >> 5);
  const long long nw = (long long)gridDim.x * kQuantWarps;
  for (long long row = w0; row < n; row += nw) {
    const float* x = X + (size_t)row * d;
    if (dtype == PEOS_BF16) {
      unsigned short* o = static_cast<unsigned short*>(out) + (size_t)row * d;
      for (int k = lane; k < d; k += 32) o[k] = __bfloat16_as_ushort(__float2bfloat16_rn(x[k]));
      if (scales && lane == 0) scales[row] = 1.0f;
      continue;
    }
    float amax = 0.0f;
    for (int k = lane; k < d; k += 32) amax = fmaxf(amax, fabsf(x[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(kFull, amax, o));
    const float sc = amax > 0.0f ? amax / 448.0f : 1.0f;
    const float inv = amax > 0.0f ? 448.0f / amax : 1.0f;
    unsigned char* o = static_cast<unsigned char*>(out) + (size_t)row * d;
    for (int k = lane; k < d; k += 32) o[k] = __nv_cvt_float_to_fp8(x[k] * inv, __NV_SATFINITE, __NV_E4M3);
    if (lane == 0) scales[row] = sc;
  }
}

}  // namespace

cudaError_t launch_quantize(const float* X, int64_t n, int d, int dtype, void* out, float* scales, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = (n + kQuantWarps - 1) / kQuantWarps;
  if (grid > (long long)sms * 8) grid = (long long)sms * 8;
  quantize_kernel<<<(unsigned)grid, kQuantWarps * 32, 0, st>>>(X, n, d, dtype, out, scales);
  return cudaGetLastError();
}

}  // namespace peos
