// Device-side building blocks of the PEOs search: the routing test, the query
// projection table, the lossy visited table and warp reductions.  Shared by the
// search kernel and the edge-statistics kernel so both run the same arithmetic.
//
// Every translation unit that includes this file is compiled with --fmad=false:
// a*b+c stays two roundings unless written as fmaf().  The test arithmetic is
// written in one fixed order (below) so that its FP32 results are reproducible.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace peos {

constexpr unsigned kFull = 0xffffffffu;
constexpr int32_t kExpanded = (int32_t)0x80000000;  // flag bit on ids stored in R
constexpr uint64_t kNoKey = ~0ull;

// Kept at six 4-byte fields: enlarging this struct (it sits inside the search
// kernel's argument block) measured 1.6x slower code for the plain kernel on sm_103a.
struct TestConst {
  float z_eps;  // Phi^{-1}(eps)
  float c_eta;  // sqrt(L) * eta
  float kL;     // L / (L + 1), in FP32 as (float)L / ((float)L + 1)
  int L, m;
  int mode;     // 0 full test, 1 only the A rules, 2 always pass
};

// outcome kinds (same numbering as the diagnostics ABI)
enum : int { kRejectA = 0, kAcceptA = 1, kDecidedH = 2, kDegenerate = 3, kNotFull = 4, kNoTest = 5 };

// Projection table of one vector x (in shared memory): t[c*m + j] = b_j . x
// (c = 0, all d dims) or a^c_j . x_c (c = 1..L, block c of d/L dims), each a
// plain sequential FP32 sum.  Entries are spread over the warp's lanes.
__device__ __forceinline__ void project_table(const float* __restrict__ x, int d, int L, int m,
                                              const float* __restrict__ A, const float* __restrict__ B,
                                              float* __restrict__ t, int lane) {
  const int dp = d / L;
  const int tw = (L + 1) * m;
  for (int e = lane; e < tw; e += 32) {
    const int c = e / m;
    const int j = e - c * m;
    float acc = 0.0f;
    if (c == 0) {
      const float* b = B + (size_t)j * d;
      for (int k = 0; k < d; ++k) acc = acc + __ldg(b + k) * x[k];
    } else {
      const int i = c - 1;
      const float* a = A + ((size_t)i * m + j) * dp;
      const float* xi = x + i * dp;
      for (int k = 0; k < dp; ++k) acc = acc + __ldg(a + k) * xi[k];
    }
    t[e] = acc;
  }
}

// The statistic's weighted sum over the table entries an edge's packed codes select:
// S(t) = w_reg * sum_{c=1..L} sgn(e[c]) t[c][|e[c]|-1] + sqrt(L) w_res * sgn(e[0]) t[0][|e[0]|-1],
// the first sum in order c = 1..L (codes: `bits` bits each, sign at bit bits - 1,
// |e[c]| - 1 below it, `cpw` codes per 64-bit word).
__device__ __forceinline__ float edge_sum(const float* __restrict__ t, const unsigned long long (&cw)[kMaxCodeWords],
                                          int bits, int cpw, float wr, float cr, int L, int m) {
  const unsigned long long mask = (1ull << bits) - 1ull;
  const int jmask = (1 << (bits - 1)) - 1;
  float h2;
  {
    const int code = (int)(cw[0] & mask);
    const float val = t[code & jmask];
    h2 = (code >> (bits - 1)) ? -val : val;
  }
  float h1 = 0.0f;
  int c = 1;
#pragma unroll
  for (int w = 0; w < kMaxCodeWords; ++w) {
    const unsigned long long word = cw[w];
    for (int k = (w == 0 ? 1 : 0); k < cpw && c <= L; ++k, ++c) {
      const int code = (int)((word >> (k * bits)) & mask);
      const float val = t[c * m + (code & jmask)];
      h1 = h1 + ((code >> (bits - 1)) ? -val : val);
    }
  }
  return wr * h1 + cr * h2;
}

// The PEOs routing test of one edge (v -> u), frame translated by -v:
//   tq       = projection table of q (shared memory); the table of x = q - v is
//              t(q) - t(v), so the statistic's sum is S(t(q)) - sv with the edge's
//              node term sv = S(t(v)) stored at index time
//   dv       = ||x||^2 (the stored exact distance of v), xn = sqrt(dv), inv = 1/xn
//   delta2   = bound of the full list
//   cw       = the edge's packed codes e[0..L]
//   en = ||e||, wr = w_reg, cr = sqrt(L) w_res
// Returns the outcome kind; `pass` says whether u goes on to the exact distance.
// The decision H >= T = A c + z sqrt(var) (z = Phi^{-1}(eps) <= 0) is taken as
// (A c - H <= 0) or ((A c - H)^2 <= z^2 var), so no square root is needed; T is
// produced only when kWantT (diagnostics).
template <bool kWantT>
__device__ __forceinline__ int peos_edge_test(const float* __restrict__ tq, float sv, float dv, float xn, float inv,
                                              float delta2, const unsigned long long (&cw)[kMaxCodeWords], int bits,
                                              int cpw, float en, float wr, float cr, const TestConst& K, bool& pass,
                                              float& A_o, float& H_o, float& T_o) {
  A_o = 0.0f;
  H_o = 0.0f;
  T_o = 0.0f;
  if (K.mode == 2) { pass = true; return kNoTest; }
  if (en == 0.0f || dv == 0.0f) { pass = true; return kDegenerate; }
  const float A = ((dv + en * en) - delta2) / (2.0f * (xn * en));
  A_o = A;
  if (A >= 1.0f) { pass = false; return kRejectA; }
  if (A <= 0.0f) { pass = true; return kAcceptA; }
  if (K.mode == 1) { pass = true; return kNoTest; }
  const float H = (edge_sum(tq, cw, bits, cpw, wr, cr, K.L, K.m) - sv) * inv;
  const float var = (wr * wr + cr * cr) - K.kL * (A * A);
  H_o = H;
  if (kWantT) T_o = A * K.c_eta + K.z_eps * sqrtf(fmaxf(var, 0.0f));
  const float g = A * K.c_eta - H;
  pass = (g <= 0.0f) || ((g * g) <= (K.z_eps * K.z_eps) * var);
  return kDecidedH;
}

// Lossy visited table: direct-mapped, slot from the top bits of a Fibonacci hash.
// A slot holding a different id means "not visited" (possibly forgotten), which
// only costs a repeated evaluation: a forgotten node is already in R or has a
// distance >= the list bound, so it never changes R.
__device__ __forceinline__ uint32_t visit_slot(int32_t id, int bits) {
  return ((uint32_t)id * 0x9E3779B1u) >> (32 - bits);
}

// (dist, id) packed so that unsigned order == lexicographic order (dist >= 0).
__device__ __forceinline__ uint64_t pack_key(float dist, int32_t id) {
  return ((uint64_t)__float_as_uint(dist) << 32) | (uint32_t)id;
}
__device__ __forceinline__ float key_dist(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ int32_t key_id(uint64_t k) { return (int32_t)(uint32_t)(k & 0xffffffffu); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ int warp_isum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

}  // namespace peos
