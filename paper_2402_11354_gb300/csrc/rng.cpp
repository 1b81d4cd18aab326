// Random projection vectors of Sec. 4.2 step (2), generated on the host.
//
// Counter-based: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11) keyed by (seed, tag), one block per four
// consecutive columns of one row of one matrix: counter = (column / 4, row,
// matrix, 0), matrix 0 = the subspace vectors a^i_j (row i*m + j), matrix 1 = the
// full-space vectors b_j (row j).  Each block's four 64-bit words become two
// Box-Muller pairs (uniforms from the top 53 bits: u1 in (0, 1], u2 in [0, 1)),
// evaluated in FP64 and rounded once to FP32.
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace peos {
namespace {

struct Philox64 {
  static constexpr uint64_t kMulA = 0xD2E7470EE14C6C93ULL;  // round multipliers
  static constexpr uint64_t kMulB = 0xCA5A826395121157ULL;
  static constexpr uint64_t kBumpA = 0x9E3779B97F4A7C15ULL;  // key schedule (Weyl) increments
  static constexpr uint64_t kBumpB = 0xBB67AE8584CAA73BULL;

  static inline void mul128(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    const unsigned __int128 p = static_cast<unsigned __int128>(a) * b;
    *hi = static_cast<uint64_t>(p >> 64);
    *lo = static_cast<uint64_t>(p);
  }

  static void block(uint64_t c[4], uint64_t k0, uint64_t k1) {
    for (int round = 0; round < 10; ++round) {
      uint64_t hA, lA, hB, lB;
      mul128(kMulA, c[0], &hA, &lA);
      mul128(kMulB, c[2], &hB, &lB);
      const uint64_t n0 = hB ^ c[1] ^ k0;
      const uint64_t n2 = hA ^ c[3] ^ k1;
      c[0] = n0;
      c[1] = lB;
      c[2] = n2;
      c[3] = lA;
      k0 += kBumpA;
      k1 += kBumpB;
    }
  }
};

constexpr uint64_t kKeyTag = 0x50454F5350524F4AULL;

void normals4(uint64_t seed, uint64_t matrix, uint64_t row, uint64_t col4, double out[4]) {
  uint64_t c[4] = {col4, row, matrix, 0};
  Philox64::block(c, seed, kKeyTag);
  const double scale = 1.0 / 9007199254740992.0;  // 2^-53
  const double tau = 6.283185307179586;
  for (int pair = 0; pair < 2; ++pair) {
    const double u1 = (static_cast<double>(c[2 * pair] >> 11) + 1.0) * scale;
    const double u2 = static_cast<double>(c[2 * pair + 1] >> 11) * scale;
    const double radius = sqrt(-2.0 * log(u1));
    const double angle = tau * u2;
    out[2 * pair] = radius * cos(angle);
    out[2 * pair + 1] = radius * sin(angle);
  }
}

}  // namespace

void projections_host(uint64_t seed, int d, int L, int m, float* A, float* B) {
  const int dp = d / L;
  double z[4];
  for (int i = 0; i < L; ++i) {
    for (int j = 0; j < m; ++j) {
      const uint64_t row = static_cast<uint64_t>(i) * static_cast<uint64_t>(m) + static_cast<uint64_t>(j);
      float* dst = A + (static_cast<size_t>(i) * m + j) * dp;
      for (int k0 = 0; k0 < dp; k0 += 4) {
        normals4(seed, 0, row, static_cast<uint64_t>(k0 / 4), z);
        for (int t = 0; t < 4 && k0 + t < dp; ++t) dst[k0 + t] = static_cast<float>(z[t]);
      }
    }
  }
  for (int j = 0; j < m; ++j) {
    float* dst = B + static_cast<size_t>(j) * d;
    for (int k0 = 0; k0 < d; k0 += 4) {
      normals4(seed, 1, static_cast<uint64_t>(j), static_cast<uint64_t>(k0 / 4), z);
      for (int t = 0; t < 4 && k0 + t < d; ++t) dst[k0 + t] = static_cast<float>(z[t]);
    }
  }
}

}  // namespace peos
