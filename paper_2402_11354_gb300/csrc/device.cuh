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
  int mode;     // 0 full test, 1 only the A rules, 2 always pass, 3 full test with the quantile table (frame Q)
};

// violation kinds counted by self-checked builds (-DPEOS_CHECKED; peos_check_read)
enum : int { kChkCandidate = 0, kChkExpanded = 1, kChkListWrite = 2, kChkOrder = 3, kChkDuplicate = 4, kChkKinds = 8 };

// outcome kinds (same numbering as the diagnostics ABI)
enum : int { kRejectA = 0, kAcceptA = 1, kDecidedH = 2, kDegenerate = 3, kNotFull = 4, kNoTest = 5 };

// Projection table of one vector x (in shared memory): t[c*m + j] = b_j . x
// (c = 0, all d dims, summed block by block: a sequential partial sum per block of d/L
// dims, then the partials in block order) or a^c_j . x_c (c = 1..L, block c of d/L dims,
// a sequential sum).  Entries are spread over the warp's lanes.
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
      for (int i = 0; i < L; ++i) {
        float part = 0.0f;
        for (int k = 0; k < dp; ++k) part = part + __ldg(b + i * dp + k) * x[i * dp + k];
        acc = acc + part;
      }
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
// the first sum in order c = 1..L.  `tf` is the sign-folded table (folded_stride): the
// code of block c indexes its signed term at (c << bits) + code.  Codes: `bits` bits each,
// `cpw` per 64-bit word; CW = the words held per edge (1 when the L + 1 codes fit one
// word, else kMaxCodeWords, unused words zero).  With one word of 5-bit codes (m <= 16,
// L <= 11) the walk is unrolled with constant shifts and block offsets: the same sums in
// the same order, 2.4% less kernel time on sift-shaped data (unrolled over three words it
// had raised register pressure and measured slower).
template <int CW>
__device__ __forceinline__ float edge_sum(const float* __restrict__ tf, const unsigned long long (&cw)[CW], int bits,
                                          int cpw, float wr, float cr, int L) {
  if (CW == 1 && bits == 5) {
    const unsigned long long w = cw[0];
    const float g2 = tf[(int)(w & 31ull)];
    float g1 = 0.0f;
#pragma unroll
    for (int c = 1; c <= 11; ++c)
      if (c <= L) g1 = g1 + tf[(c << 5) | (int)((w >> (5 * c)) & 31ull)];
    return wr * g1 + cr * g2;
  }
  const unsigned long long mask = (1ull << bits) - 1ull;
  const float h2 = tf[(int)(cw[0] & mask)];
  float h1 = 0.0f;
  int c = 1;
#pragma unroll
  for (int w = 0; w < CW; ++w) {
    const unsigned long long word = cw[w];
    for (int k = (w == 0 ? 1 : 0); k < cpw && c <= L; ++k, ++c)
      h1 = h1 + tf[(c << bits) | (int)((word >> (k * bits)) & mask)];
  }
  return wr * h1 + cr * h2;
}

// Sign-folded projection table of x written straight into tf (folded_stride): the same
// sequential FP32 sums as project_table, each entry stored as itself and negated.
__device__ __forceinline__ void project_table_folded(const float* __restrict__ x, int d, int L, int m, int bits,
                                                     const float* __restrict__ A, const float* __restrict__ B,
                                                     float* __restrict__ tf, int lane) {
  const int dp = d / L;
  const int tw = (L + 1) * m;
  const int half = 1 << (bits - 1);
  for (int e = lane; e < tw; e += 32) {
    const int c = e / m;
    const int j = e - c * m;
    float acc = 0.0f;
    if (c == 0) {
      const float* b = B + (size_t)j * d;
      for (int i = 0; i < L; ++i) {
        float part = 0.0f;
        for (int k = 0; k < dp; ++k) part = part + __ldg(b + i * dp + k) * x[i * dp + k];
        acc = acc + part;
      }
    } else {
      const int i = c - 1;
      const float* a = A + ((size_t)i * m + j) * dp;
      const float* xi = x + i * dp;
      for (int k = 0; k < dp; ++k) acc = acc + __ldg(a + k) * xi[k];
    }
    tf[(c << bits) + j] = acc;
    tf[(c << bits) + half + j] = -acc;
  }
}

// The same table from the k-major copy Wt (element (t, j) of B^T at t m + j, of the a^i
// at d m + t m + j with t = (i - 1) d' + k), for m <= 16: lane j < 16 forms entry (0, j)
// = b_j . x and lane 16 + j the entries (c, j), c = 1..L.  Both halves walk the blocks of
// the space partition together (both read the same x[t]): per block a fused
// multiply-add chain over its d' coordinates, after which lanes 16 + j store entry
// (c, j) and lanes j add the block's partial sum into entry (0, j).
__device__ __forceinline__ void project_table_folded_kmajor(const float* __restrict__ x, int d, int L, int m,
                                                            int bits, const float* __restrict__ Wt,
                                                            float* __restrict__ tf, int lane) {
  const int dp = d / L;
  const int half = 1 << (bits - 1);
  const int j = lane & 15;
  const bool isB = lane < 16;
  if (j >= m) return;
  const float* w = Wt + (isB ? 0 : (size_t)d * m) + j;
  float tot = 0.0f;
  for (int i = 0; i < L; ++i) {
    float acc = 0.0f;
    const float* wi = w + (size_t)i * dp * m;
    const float* xi = x + i * dp;
#pragma unroll 4
    for (int k = 0; k < dp; ++k) acc = fmaf(wi[(size_t)k * m], xi[k], acc);
    if (isB) {
      tot = tot + acc;
    } else {
      tf[((i + 1) << bits) + j] = acc;
      tf[((i + 1) << bits) + half + j] = -acc;
    }
  }
  if (isB) {
    tf[j] = tot;
    tf[half + j] = -tot;
  }
}

// Sign-folded copy of a table t ((L+1)*m entries) into tf (folded_stride), warp-wide.
__device__ __forceinline__ void fold_table(const float* __restrict__ t, int L, int m, int bits,
                                           float* __restrict__ tf, int lane) {
  const int half = 1 << (bits - 1);
  for (int e = lane; e < (L + 1) * m; e += 32) {
    const int c = e / m, j = e - c * m;
    tf[(c << bits) + j] = t[e];
    tf[(c << bits) + half + j] = -t[e];
  }
}

// The PEOs routing test of one edge (v -> u), frame translated by -v:
//   tf       = the sign-folded projection table of q (shared memory); the table of
//              x = q - v is t(q) - t(v), so the statistic's sum is S(t(q)) - sv with the
//              edge's node term sv = S(t(v)) stored at index time
//   dv       = ||x||^2 (the stored exact distance of v), xn = sqrt(dv), inv = 1/xn
//   delta2   = bound of the full list
//   cw       = the edge's packed codes e[0..L]
//   en = ||e||, wr = w_reg, cr = sqrt(L) w_res
// Returns the outcome kind; `pass` says whether u goes on to the exact distance.
// The decision H >= T = A c + z sqrt(var) (z = Phi^{-1}(eps) <= 0) is taken as
// (A c - H <= 0) or ((A c - H)^2 <= z^2 var), so no square root is needed; T is
// produced only when kWantT (diagnostics).
template <bool kWantT, int CW>
__device__ __forceinline__ int peos_edge_test(const float* __restrict__ tf, float sv, float dv, float xn, float inv,
                                              float delta2, const unsigned long long (&cw)[CW], int bits,
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
  const float H = (edge_sum(tf, cw, bits, cpw, wr, cr, K.L) - sv) * inv;
  const float var = (wr * wr + cr * cr) - K.kL * (A * A);
  H_o = H;
  if (kWantT) T_o = A * K.c_eta + K.z_eps * sqrtf(fmaxf(var, 0.0f));
  const float g = A * K.c_eta - H;
  pass = (g <= 0.0f) || ((g * g) <= (K.z_eps * K.z_eps) * var);
  return kDecidedH;
}

// The PEOs test in the paper-literal frame Q: tf is the sign-folded table of q' = q/||q||;
// A = ((||u||^2/2 - r) - v.q) / (||q|| ||e||) (Eq. A_r), the inner products formed by the
// caller from distances and squared norms; the rest as in peos_edge_test, with H read
// straight from the table (no node term).
template <int CW>
__device__ __forceinline__ int peos_edge_test_q(const float* __restrict__ tf, float vq, float r, float un2, float qn,
                                                const unsigned long long (&cw)[CW], int bits, int cpw,
                                                float en, float wr, float cr, const TestConst& K, bool& pass) {
  if (K.mode == 2) { pass = true; return kNoTest; }
  if (en == 0.0f || qn == 0.0f) { pass = true; return kDegenerate; }
  const float A = ((un2 / 2.0f - r) - vq) / (qn * en);
  if (A >= 1.0f) { pass = false; return kRejectA; }
  if (A <= 0.0f) { pass = true; return kAcceptA; }
  if (K.mode == 1) { pass = true; return kNoTest; }
  const float H = edge_sum(tf, cw, bits, cpw, wr, cr, K.L);
  float var = (wr * wr + cr * cr) - K.kL * (A * A);
  if (K.mode == 3) {
    // the quantile table of Sec. 4.3: 0 <= var <= L on 256 L bins of width 1/256, the
    // bin's upper edge (a slightly smaller quantile, z < 0)
    int bin = (int)(var * 256.0f);
    bin = bin < 0 ? 0 : (bin > 256 * K.L - 1 ? 256 * K.L - 1 : bin);
    var = (float)(bin + 1) * (1.0f / 256.0f);
  }
  const float g = A * K.c_eta - H;
  pass = (g <= 0.0f) || ((g * g) <= (K.z_eps * K.z_eps) * var);
  return kDecidedH;
}

// The SimHash test of the residual remedy (Sec. 3.1, Lemma 4.1), frame translated by -v:
// the same A rules as the PEOs test, then pass iff A <= acrit[#Col] with
// #Col = K - popcount(bits(e) xor bits(x)) (the thresholds are tabulated on the host).
template <int CW>
__device__ __forceinline__ int simhash_edge_test(const float* __restrict__ acrit, int K, int words,
                                                 const unsigned long long (&bx)[CW],
                                                 const unsigned long long (&cw)[CW], float dv, float xn,
                                                 float delta2, float en, int mode, bool& pass) {
  if (mode == 2) { pass = true; return kNoTest; }
  if (en == 0.0f || dv == 0.0f) { pass = true; return kDegenerate; }
  const float A = ((dv + en * en) - delta2) / (2.0f * (xn * en));
  if (A >= 1.0f) { pass = false; return kRejectA; }
  if (A <= 0.0f) { pass = true; return kAcceptA; }
  if (mode == 1) { pass = true; return kNoTest; }
  int diff = 0;
#pragma unroll
  for (int w = 0; w < CW; ++w)
    if (w < words) diff += __popcll(cw[w] ^ bx[w]);
  pass = A <= acrit[K - diff];
  return kDecidedH;
}

// Lossy visited table: direct-mapped, slot from the top bits of a Fibonacci hash.
// A slot holding a different id means "not visited" (possibly forgotten), which
// only costs a repeated evaluation: a forgotten node is already in R or has a
// distance >= the list bound, so it never changes R.
__device__ __forceinline__ uint32_t visit_slot(int32_t id, int bits) {
  return ((uint32_t)id * 0x9E3779B1u) >> (32 - bits);
}
__device__ __forceinline__ bool visit_seen(const int32_t* vis, int32_t id, int bits) {
  return vis[visit_slot(id, bits)] == id;
}
__device__ __forceinline__ void visit_mark(int32_t* vis, int32_t id, int bits) { vis[visit_slot(id, bits)] = id; }

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
