// Device-memory layouts shared by the host launchers and the kernels.
#pragma once
#include <stddef.h>

#ifdef __CUDACC__
#define PEOS_HD __host__ __device__
#else
#define PEOS_HD
#endif

namespace peos {

constexpr int kMaxEf = 1024;  // largest result list (efs)
constexpr int kMaxR = 64;     // largest out-degree

// Packed extreme-value codes: code e[c] (c = 0..L) of an edge is stored in code_bits(m)
// bits as (|e[c]| - 1) | (e[c] < 0) << (bits - 1); codes_per_word(m) codes fill one
// 64-bit word from the low bits up; an edge has code_words(L, m) <= kMaxCodeWords words.
constexpr int kMaxCodeWords = 3;
PEOS_HD inline int code_bits(int m) {
  int b = 1;
  while ((1 << b) < m) ++b;
  return b + 1;
}
PEOS_HD inline int codes_per_word(int m) { return 64 / code_bits(m); }
PEOS_HD inline int code_words(int L, int m) { return (L + 1 + codes_per_word(m) - 1) / codes_per_word(m); }

// Edge record of a node (R edges), every field an array over the edges:
//   scalars          at byte 0, in one of three forms (`sbits`, the scalar width):
//                      32: float4 (||e||, w_reg, sqrt(L) w_res, sv)[R]
//                      16: float4 step, float sv[R], short4 q[R] at rec_q_offset(R)
//                       8: float4 step, {char4 q, float sv}[R] at rec_pair_offset()
//                          (a lane reads its edge's scalars and node term in one 8-byte load)
//                    (compact forms: step = the node's quantisation steps of ||e||, w_reg,
//                    sqrt(L) w_res (4th unused); q = (q_e, q_w, q_c, 0), the scalar read
//                    as (float) q * step; sv stays FP32, computed from those scalars)
//   int32  ids[R]    at rec_ids_offset(R, sbits)
//   uint64 codes[W][R] at rec_codes_offset(R, sbits), 16-byte aligned
// padded to 32 bytes; sv = the edge's node term S(t(v)) of the statistic.
PEOS_HD inline size_t rec_sv_offset(int /*R*/) { return 16; }                                  // 16-bit form
PEOS_HD inline size_t rec_q_offset(int R) { return (16 + (size_t)4 * R + 7) & ~(size_t)7; }  // 16-bit form
PEOS_HD inline size_t rec_pair_offset() { return 16; }                                        // 8-bit form
PEOS_HD inline size_t rec_scalar_bytes(int R, int sbits) {
  return sbits == 32 ? (size_t)16 * R : sbits == 16 ? rec_q_offset(R) + (size_t)8 * R : rec_pair_offset() + (size_t)8 * R;
}
PEOS_HD inline size_t rec_ids_offset(int R, int sbits = 32) { return rec_scalar_bytes(R, sbits); }
PEOS_HD inline size_t rec_codes_offset(int R, int sbits = 32) {
  return (rec_ids_offset(R, sbits) + (size_t)4 * R + 15) & ~(size_t)15;
}
PEOS_HD inline size_t record_stride_words(int R, int words, int sbits = 32) {
  size_t b = rec_codes_offset(R, sbits) + (size_t)8 * words * R;
  return (b + 31) & ~(size_t)31;
}
PEOS_HD inline size_t record_stride(int R, int L, int m, int sbits = 32) {
  return record_stride_words(R, code_words(L, m), sbits);
}

// SimHash records (the baseline test of Sec. 3.1) use the same layout: scal = (||e||, 0,
// 0, 0) and K sign bits in K / 64 words (bit i of the edge in word i / 64 at i % 64).
constexpr int kMaxSimHashBits = 64 * kMaxCodeWords;

// Node projection table row: (L+1)*m floats padded to a multiple of 4 (16-byte rows).
PEOS_HD inline int table_stride(int L, int m) { return ((L + 1) * m + 3) & ~3; }

// Sign-folded query table, the form the search reads: block c holds 2^bits floats,
// entry (c, j) at c * 2^bits + j and its negation at c * 2^bits + 2^(bits-1) + j, so a
// packed code (|e[c]| - 1, sign in bit bits - 1) indexes its signed term directly.
// Entries with j >= m are never read.
PEOS_HD inline int folded_stride(int L, int m) { return (((L + 1) << code_bits(m)) + 3) & ~3; }

}  // namespace peos
