/*
 * PEOs oracle: a plain, slow, CPU reference of the PEOs routing hot path
 * (Probabilistic Routing for Graph-Based ANNS, arXiv 2402.11354).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the tests, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py load it.  It shares no code with the CUDA path.
 *
 * Arithmetic conventions (the paper fixes no precision, so these are readings):
 *   - everything the method computes is FP32, evaluated in the plain sequential
 *     order written below; this file must be compiled with -ffp-contract=off so
 *     that a*b+c is two roundings, exactly as written;
 *   - reference distances (ground truth, graph construction) are FP64;
 *   - random projection vectors come from Philox4x64-10 + Box-Muller in FP64,
 *     rounded once to FP32.
 *
 * Functions and the passages they follow:
 *   orc_philox4x64_10 .. counter-based generator (Salmon et al., SC'11)
 *   orc_projections ..... Sec. 4.2 step (2): a^i_j ~ N(0, I_{d'}), b_j ~ N(0, I_d)
 *   orc_build_codes ..... Sec. 4.2 steps (1) and (3): e = e_reg + e_res, w_reg, w_res,
 *                         extreme-value codes e[0..L]
 *   orc_quantize ........ the precision form's storage of the base rows: BF16 (round to
 *                         nearest even) and FP8-E4M3 with a per-row scale max|x| / 448
 *   orc_quantize_scalars  the compact index's 8/16-bit edge scalars (Sec. 4.3 space analysis,
 *                         Sec. 6.4 PEOs (Compact)): per-node linear steps, round half to even
 *   orc_project, orc_node_proj
 *                         the projection table of Sec. 4.3 / Algorithm 2 (T_I) of one vector:
 *                         its inner products with every a^i_j and b_j, plain sequential sums
 *   orc_dim_permutation . Appendix D.1: balanced assignment of coordinates to subspaces;
 *                         with a permutation the codes and tables are of the permuted
 *                         vectors, exact distances of the stored ones
 *   orc_norm_ppf, orc_eta  the quantile F^{-1} of Eq. (N_ex_min), Sec. 4.2 step (4)
 *   orc_edge_stats ...... Sec. 4.2 steps (5)-(6), Eq. (A_r), Eq. (criterion), Algorithm 2,
 *                         for the out-edges of one node
 *   orc_search .......... Algorithm 1 (graph ANNS with routing), plain or with the PEOs test
 *   orc_simhash_build, orc_simhash_acrit
 *                         the SimHash test of Sec. 3.1 / Lemma 4.1 with the residual remedy
 *                         and a Hoeffding threshold (a baseline of the routing tests)
 *   orc_greedy_layer .... the hierarchical entry of the paper's HNSW indexes (Sec. 6.1): greedy
 *                         descent with a list of one through each upper layer
 *   orc_knn_f64 ......... Definition of NNS / K-NN (Sec. 2), brute force in FP64
 *   orc_build_graph ..... the proximity graph G=(V,E) of Sec. 2: exact kNN candidates,
 *                         relative-neighbourhood pruning, reverse edges, connectivity repair
 *
 * The routing test is evaluated the way Sec. 4.2 states it, with nothing precomputed
 * beyond what steps (1)-(3) name: in the frame translated by -v (the default) the
 * query vector of an expansion of v is x = q - v; it is normalised to x' = x / ||x||,
 * projected onto every a^i_j and b_j (the table of step 5, sequential sums over the
 * dimensions), H = w_reg H_1 + sqrt(L) w_res H_2 is read from that table, T = A sqrt(2 L
 * ln m) + Phi^{-1}(eps) sqrt(var) is the eps-quantile of Eq. (N_ex_min), and the edge
 * passes iff H - T >= 0 (Eq. criterion).  In the paper-literal frame Q the table is that
 * of q' = q / ||q||, built once per query, and A_r of Eq. (A_r) uses plain FP32 dot
 * products.  The visited set is exact.
 *
 * Every function above is pinned by tests/test_oracle_*.py against something outside
 * this file (definitions in FP64, closed forms, values the paper prints, examples
 * worked by hand, numpy's Philox and torch's conversions, brute force); the pins are
 * themselves checked by compiling copies of this file with planted mistakes, each of
 * which must fail one of them (tests/test_oracle_mutations.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_E_INVAL 1
#define ORC_E_NOMEM 2
#define ORC_E_OVERFLOW 4

/* ------------------------------------------------------------------------- */
/* Philox4x64-10                                                              */
/* ------------------------------------------------------------------------- */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL;
/* second key word: fixed tag so that a seed alone keys the generator */
static const uint64_t PEOS_KEY_TAG = 0x50454F5350524F4AULL;

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
    unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Four standard normals for columns 4g..4g+3 of row `row` of matrix `mat`
 * (mat 0 = the subspace vectors a^i_j, mat 1 = the full-space vectors b_j).
 * Two Box-Muller pairs, each from two 53-bit uniforms. */
static void gauss4(uint64_t seed, uint64_t mat, uint64_t row, uint64_t g, double z[4]) {
  uint64_t ctr[4] = {g, row, mat, 0};
  uint64_t key[2] = {seed, PEOS_KEY_TAG};
  uint64_t w[4];
  orc_philox4x64_10(ctr, key, w);
  const double two_m53 = 1.0 / 9007199254740992.0; /* 2^-53 */
  const double two_pi = 6.283185307179586;
  for (int h = 0; h < 2; ++h) {
    double u1 = ((double)(w[2 * h] >> 11) + 1.0) * two_m53; /* (0, 1] */
    double u2 = (double)(w[2 * h + 1] >> 11) * two_m53;      /* [0, 1) */
    double r = sqrt(-2.0 * log(u1));
    double th = two_pi * u2;
    z[2 * h] = r * cos(th);
    z[2 * h + 1] = r * sin(th);
  }
}

/* Sec. 4.2 step (2).  A is [L][m][d'] row-major, B is [m][d] row-major. */
int orc_projections(uint64_t seed, int d, int L, int m, float* A, float* B) {
  if (d <= 0 || L <= 0 || m <= 0 || d % L != 0) return ORC_E_INVAL;
  int dp = d / L;
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < m; ++j) {
      uint64_t row = (uint64_t)i * (uint64_t)m + (uint64_t)j;
      for (int k = 0; k < dp; ++k) {
        double z[4];
        gauss4(seed, 0, row, (uint64_t)(k / 4), z);
        A[((size_t)i * m + j) * dp + k] = (float)z[k % 4];
      }
    }
  for (int j = 0; j < m; ++j)
    for (int k = 0; k < d; ++k) {
      double z[4];
      gauss4(seed, 1, (uint64_t)j, (uint64_t)(k / 4), z);
      B[(size_t)j * d + k] = (float)z[k % 4];
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Reduced-precision storage of the base vectors                              */
/* ------------------------------------------------------------------------- */
/* bfloat16: the upper 16 bits of the IEEE binary32 pattern, rounded to nearest
 * even on the dropped 16 bits (NaN kept quiet). */
static uint16_t f32_to_bf16(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}

static float bf16_to_f32(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float x;
  memcpy(&x, &u, 4);
  return x;
}

/* FP8 E4M3 (OCP 8-bit floating point, "E4M3FN"): 1 sign bit, 4 exponent bits (bias 7),
 * 3 mantissa bits; no infinities; largest finite 448; subnormals 2^-6 * m/8.  Values
 * are rounded to the nearest representable one, ties to even, and magnitudes beyond
 * 448 saturate to 448. */
static float e4m3_value(int code) {
  int sgn = (code >> 7) & 1, ex = (code >> 3) & 15, man = code & 7;
  float v = (ex == 0) ? ldexpf((float)man / 8.0f, -6) : ldexpf(1.0f + (float)man / 8.0f, ex - 7);
  return sgn ? -v : v;
}

/* The 127 non-negative finite values in code order (ascending). */
static float g_e4m3_pos[127];
static void e4m3_table(void) {
  for (int c = 0; c < 127; ++c) g_e4m3_pos[c] = e4m3_value(c);
}

static uint8_t f32_to_e4m3(float x) {
  int neg = signbit(x) ? 1 : 0;
  float a = fabsf(x);
  if (a >= 448.0f) return (uint8_t)((neg << 7) | 0x7e);  /* saturate to 448 */
  /* bracket a between two consecutive values, then take the nearer one, ties to the
   * even code */
  int lo = 0, hi = 126;
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (g_e4m3_pos[mid] <= a) lo = mid; else hi = mid;
  }
  float dl = a - g_e4m3_pos[lo], dh = g_e4m3_pos[hi] - a;
  int best = (dl < dh) ? lo : (dh < dl) ? hi : ((lo & 1) == 0 ? lo : hi);
  return (uint8_t)((neg << 7) | best);
}

/* Quantise rows of X: dtype 1 = bf16 (scales all 1), 2 = e4m3 with a per-row scale
 * s = max|x| / 448 (1 for an all-zero row), codes of x * (448 / max|x|).  Writes the
 * codes (2 or 1 bytes per element), the scales, and the dequantised values
 * deq = s * value(code) in FP32. */
int orc_quantize(const float* X, int64_t n, int d, int dtype, void* codes, float* scales, float* deq) {
  if (dtype != 1 && dtype != 2) return ORC_E_INVAL;
  e4m3_table();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const float* x = X + (size_t)i * d;
    if (dtype == 1) {
      uint16_t* c = (uint16_t*)codes + (size_t)i * d;
      for (int k = 0; k < d; ++k) {
        c[k] = f32_to_bf16(x[k]);
        deq[(size_t)i * d + k] = bf16_to_f32(c[k]);
      }
      scales[i] = 1.0f;
    } else {
      uint8_t* c = (uint8_t*)codes + (size_t)i * d;
      float amax = 0.0f;
      for (int k = 0; k < d; ++k) amax = fmaxf(amax, fabsf(x[k]));
      float sc = amax > 0.0f ? amax / 448.0f : 1.0f;
      float inv = amax > 0.0f ? 448.0f / amax : 1.0f;
      for (int k = 0; k < d; ++k) {
        c[k] = f32_to_e4m3(x[k] * inv);
        deq[(size_t)i * d + k] = sc * e4m3_value(c[k]);
      }
      scales[i] = sc;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Normal quantile and eta                                                    */
/* ------------------------------------------------------------------------- */
static double norm_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Phi^{-1}(p) by bisection on Phi to full double resolution. */
double orc_norm_ppf(double p) {
  if (!(p > 0.0 && p < 1.0)) return NAN;
  double lo = -40.0, hi = 40.0;
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (norm_cdf(mid) < p) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* eta of Lemma 4.2: mode 0 -> sqrt(2 ln m) (the paper's asymptotic value);
 * mode 1 -> E[max_j |g_j|] for m iid N(0,1), i.e. int_0^inf 1 - erf(x/sqrt2)^m dx,
 * by composite Simpson on [0, 40]. */
double orc_eta(int m, int mode) {
  if (m < 2) return NAN;
  if (mode == 0) return sqrt(2.0 * log((double)m));
  const int nint = 400000;
  const double a = 0.0, b = 40.0, h = (b - a) / nint;
  double s = 0.0;
  for (int i = 0; i <= nint; ++i) {
    double x = a + h * i;
    double f = 1.0 - pow(erf(x / sqrt(2.0)), (double)m);
    double w = (i == 0 || i == nint) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    s += w * f;
  }
  return s * h / 3.0;
}

/* ------------------------------------------------------------------------- */
/* Code builder, Sec. 4.2 steps (1) and (3)                                   */
/* ------------------------------------------------------------------------- */
/* Edge record of edge (v -> u): codes[c] for c = 0..L (c = 0 is e[0] over the
 * b_j with e_res; c = i >= 1 is e[i] over the a^i_j with e_i), stored as the
 * signed 1-based index sgn * (j + 1).  Ties in |projection| take the lowest j;
 * sgn(0) = +1.  enorm = ||e||, wreg = w_reg, cres = sqrt(L) w_res with
 * w_res = sqrt(max(0, 1 - w_reg^2)) (w_reg^2 + w_res^2 = 1 since e_reg is
 * orthogonal to e_res). */
static int argmax_abs(const float* p, int m) {
  int best = 0;
  float bv = fabsf(p[0]);
  for (int j = 1; j < m; ++j) {
    float a = fabsf(p[j]);
    if (a > bv) { bv = a; best = j; }
  }
  return best;
}

static void build_edge(const float* xv, const float* xu, int d, int L, int m,
                       const float* A, const float* B, float* e, float* eres, float* p,
                       float* bn, int8_t* codes, float* enorm, float* wreg, float* cres) {
  int dp = d / L;
  for (int k = 0; k < d; ++k) e[k] = xu[k] - xv[k];
  float tot2 = 0.0f, s = 0.0f;
  for (int i = 0; i < L; ++i) {
    float n2 = 0.0f;
    for (int k = 0; k < dp; ++k) { float t = e[i * dp + k]; n2 = n2 + t * t; }
    bn[i] = sqrtf(n2);
    tot2 = tot2 + n2;
    s = s + bn[i];
  }
  float en = sqrtf(tot2);
  *enorm = en;
  if (en == 0.0f) { /* duplicate vectors: degenerate edge, always passes the test */
    for (int c = 0; c <= L; ++c) codes[c] = 1;
    *wreg = 1.0f;
    *cres = 0.0f;
    return;
  }
  float w = s / (sqrtf((float)L) * en);
  if (w > 1.0f) w = 1.0f;
  *wreg = w;
  *cres = sqrtf((float)L) * sqrtf(fmaxf(0.0f, 1.0f - w * w)); /* sqrt(L) w_res, w_res^2 = 1 - w_reg^2 */
  float mean_bn = s / (float)L;
  for (int i = 0; i < L; ++i) {
    float coef = (bn[i] > 0.0f) ? (1.0f - mean_bn / bn[i]) : 0.0f;
    for (int k = 0; k < dp; ++k) eres[i * dp + k] = e[i * dp + k] * coef;
  }
  /* e[i], i = 1..L: argmax_j |e_i . a^i_j| */
  for (int i = 0; i < L; ++i) {
    for (int j = 0; j < m; ++j) {
      const float* a = A + ((size_t)i * m + j) * dp;
      float acc = 0.0f;
      for (int k = 0; k < dp; ++k) acc = acc + a[k] * e[i * dp + k];
      p[j] = acc;
    }
    int jb = argmax_abs(p, m);
    codes[i + 1] = (int8_t)((p[jb] >= 0.0f) ? (jb + 1) : -(jb + 1));
  }
  /* e[0]: argmax_j |e_res . b_j| */
  for (int j = 0; j < m; ++j) {
    const float* b = B + (size_t)j * d;
    float acc = 0.0f;
    for (int k = 0; k < d; ++k) acc = acc + b[k] * eres[k];
    p[j] = acc;
  }
  int jb = argmax_abs(p, m);
  codes[0] = (int8_t)((p[jb] >= 0.0f) ? (jb + 1) : -(jb + 1));
}

/* Codes of all out-edges of node v.  Layout: codes[(v*R + s)*(L+1) + c],
 * enorm[v*R + s], wreg[v*R + s], cres[v*R + s].  Empty slots (id < 0) get codes 0 and
 * zero scalars. */
static void build_node(const float* X, int d, const int32_t* nbrs, int R, int L, int m,
                       const float* A, const float* B, int64_t v, int8_t* codes,
                       float* enorm, float* wreg, float* cres, float* scratch) {
  float* e = scratch;
  float* eres = e + d;
  float* bn = eres + d;
  float* p = bn + L;
  for (int s = 0; s < R; ++s) {
    size_t es = (size_t)v * R + s;
    int32_t u = nbrs[es];
    if (u < 0) {
      memset(codes + es * (L + 1), 0, (size_t)(L + 1));
      enorm[es] = 0.0f;
      wreg[es] = 0.0f;
      cres[es] = 0.0f;
      continue;
    }
    build_edge(X + (size_t)v * d, X + (size_t)u * d, d, L, m, A, B, e, eres, p, bn,
               codes + es * (L + 1), enorm + es, wreg + es, cres + es);
  }
}

int orc_build_codes(const float* X, int64_t n, int d, const int32_t* nbrs, int R, int L, int m,
                    const float* A, const float* B, int8_t* codes, float* enorm, float* wreg, float* cres) {
  if (n < 0 || d <= 0 || L <= 0 || d % L != 0 || m < 2 || m > 127 || R <= 0) return ORC_E_INVAL;
  int fail = 0;
#pragma omp parallel
  {
    float* scratch = (float*)malloc(sizeof(float) * (size_t)(2 * d + L + m));
    if (!scratch) {
#pragma omp atomic write
      fail = 1;
    } else {
#pragma omp for schedule(dynamic, 64)
      for (int64_t v = 0; v < n; ++v)
        build_node(X, d, nbrs, R, L, m, A, B, v, codes, enorm, wreg, cres, scratch);
      free(scratch);
    }
  }
  return fail ? ORC_E_NOMEM : ORC_OK;
}

/* Scalar quantisation of the compact index (Sec. 4.3's space analysis and Sec. 6.4's
 * PEOs (Compact): every edge scalar stored in 8 or 16 bits; the paper fixes no scheme, so
 * this is a reading): per node v and per scalar kind (||e||, w_reg, sqrt(L) w_res), over
 * v's valid edges,
 *   s = max |x|,  step = s / Qb (FP32 division, Qb = 2^(bits-1) - 1),
 *   q = rint(x / step) clamped to [-Qb, Qb] (0 when step = 0),  x' = (float) q * step,
 * round half to even.  The arrays are replaced by x' in place (the test then uses x'
 * wherever it uses the scalar); steps[v*3 + kind] and qv[(v*R + s)*3 + kind] receive the
 * stored values (either may be NULL).  Empty slots keep x' = q = 0. */
int orc_quantize_scalars(int64_t n, const int32_t* nbrs, int R, int bits, float* enorm, float* wreg, float* cres,
                         float* steps, int32_t* qv) {
  if (n < 0 || R <= 0 || (bits != 8 && bits != 16)) return ORC_E_INVAL;
  const float Qb = (float)((1 << (bits - 1)) - 1);
  float* arr[3] = {enorm, wreg, cres};
  for (int64_t v = 0; v < n; ++v) {
    for (int k = 0; k < 3; ++k) {
      float* x = arr[k] + (size_t)v * R;
      float smax = 0.0f;
      for (int s = 0; s < R; ++s)
        if (nbrs[(size_t)v * R + s] >= 0 && fabsf(x[s]) > smax) smax = fabsf(x[s]);
      const float step = smax / Qb;
      if (steps) steps[(size_t)v * 3 + k] = step;
      for (int s = 0; s < R; ++s) {
        int32_t q = 0;
        if (nbrs[(size_t)v * R + s] >= 0 && step > 0.0f) {
          float r = rintf(x[s] / step);
          if (r > Qb) r = Qb;
          if (r < -Qb) r = -Qb;
          q = (int32_t)r;
        }
        x[s] = (float)q * step;
        if (qv) qv[((size_t)v * R + s) * 3 + k] = q;
      }
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Projection table of one vector (Algorithm 2's T_I, written per vector)     */
/* ------------------------------------------------------------------------- */
/* t[c*m + j]: c = 0 -> b_j . x over all d dims; c = i >= 1 -> a^i_j . x_i over block i
 * (x_i = coordinates (i-1) d' .. i d' - 1 of x).  Every entry is a plain sequential FP32
 * sum over its dimensions. */
void orc_project(const float* x, int d, int L, int m, const float* A, const float* B, float* t) {
  int dp = d / L;
  for (int j = 0; j < m; ++j) {
    const float* b = B + (size_t)j * d;
    float acc = 0.0f;
    for (int k = 0; k < d; ++k) acc = acc + b[k] * x[k];
    t[j] = acc;
  }
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < m; ++j) {
      const float* a = A + ((size_t)i * m + j) * dp;
      float acc = 0.0f;
      for (int k = 0; k < dp; ++k) acc = acc + a[k] * x[i * dp + k];
      t[(size_t)(i + 1) * m + j] = acc;
    }
}

int orc_node_proj(const float* X, int64_t n, int d, int L, int m, const float* A, const float* B, float* T) {
  if (d % L != 0) return ORC_E_INVAL;
  size_t tw = (size_t)(L + 1) * m;
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) orc_project(X + (size_t)v * d, d, L, m, A, B, T + (size_t)v * tw);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Dimension permutation (Appendix D.1)                                       */
/* ------------------------------------------------------------------------- */
/* Avg(e_j) = sum over the edges of (e_j)^2 / |E| for every coordinate j (FP64); the
 * coordinates in ascending order of Avg (ties: lower j first); then d/L rounds: round l
 * hands its L coordinates, in that order, each to the subspace with the greatest running
 * sum of Avg among those not yet served this round (ties: lower subspace index).
 * perm[i*d' + t] = the t-th coordinate given to subspace i: coordinate t of block i of a
 * permuted vector is coordinate perm[i*d' + t] of the original. */
typedef struct { double v; int j; } dimval;
static int cmp_dimval(const void* a, const void* b) {
  const dimval* x = (const dimval*)a;
  const dimval* y = (const dimval*)b;
  if (x->v < y->v) return -1;
  if (x->v > y->v) return 1;
  return (x->j > y->j) - (x->j < y->j);
}

int orc_dim_permutation(const float* X, int64_t n, int d, const int32_t* nbrs, int R, int L, int32_t* perm) {
  if (L <= 0 || d % L != 0) return ORC_E_INVAL;
  int dp = d / L;
  double* sum = (double*)calloc((size_t)d, sizeof(double));
  dimval* order = (dimval*)malloc(sizeof(dimval) * (size_t)d);
  double* load = (double*)calloc((size_t)L, sizeof(double));
  int* cnt = (int*)calloc((size_t)L, sizeof(int));
  char* served = (char*)malloc((size_t)L);
  if (!sum || !order || !load || !cnt || !served) {
    free(sum); free(order); free(load); free(cnt); free(served);
    return ORC_E_NOMEM;
  }
  int64_t ne = 0;
  for (int64_t v = 0; v < n; ++v)
    for (int s = 0; s < R; ++s) {
      int32_t u = nbrs[(size_t)v * R + s];
      if (u < 0) continue;
      ++ne;
      for (int j = 0; j < d; ++j) {
        double e = (double)X[(size_t)u * d + j] - (double)X[(size_t)v * d + j];
        sum[j] += e * e;
      }
    }
  for (int j = 0; j < d; ++j) {
    order[j].v = ne ? sum[j] / (double)ne : 0.0;
    order[j].j = j;
  }
  qsort(order, (size_t)d, sizeof(dimval), cmp_dimval);
  for (int l = 0; l < dp; ++l) {
    memset(served, 0, (size_t)L);
    for (int t = 0; t < L; ++t) {
      const dimval* dv = &order[l * L + t];
      int best = -1;
      for (int i = 0; i < L; ++i)
        if (!served[i] && (best < 0 || load[i] > load[best])) best = i;
      served[best] = 1;
      load[best] += dv->v;
      perm[best * dp + cnt[best]] = dv->j;
      ++cnt[best];
    }
  }
  free(sum); free(order); free(load); free(cnt); free(served);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Distances                                                                  */
/* ------------------------------------------------------------------------- */
/* squared l2 distance in FP32, sequential order */
float orc_dist2_f32(const float* a, const float* b, int d) {
  float acc = 0.0f;
  for (int k = 0; k < d; ++k) { float t = a[k] - b[k]; acc = acc + t * t; }
  return acc;
}

static float dot_f32(const float* a, const float* b, int d) {
  float acc = 0.0f;
  for (int k = 0; k < d; ++k) acc = acc + a[k] * b[k];
  return acc;
}

static double dist2_f64(const float* a, const float* b, int d) {
  double acc = 0.0;
  for (int k = 0; k < d; ++k) { double t = (double)a[k] - (double)b[k]; acc += t * t; }
  return acc;
}

/* ------------------------------------------------------------------------- */
/* PEOs routing test, Sec. 4.2 steps (5)-(6) and Algorithm 2                  */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t k, ef;
  int32_t routing;        /* 0 plain (every unvisited neighbour is evaluated), 1 PEOs, 2 SimHash */
  int32_t test_mode;      /* 0 full test, 1 cut-only (T = -inf), 2 always pass, 3 full test with the
                             quantile table (frame Q) */
  int32_t frame;          /* 0 = frame T (translate by -v), 1 = frame Q (paper-literal A_r) */
  int32_t max_expansions; /* safety cap per query */
  int32_t trace_cap;      /* expansions recorded per query (0 = none) */
  float z_eps;            /* Phi^{-1}(eps) */
  float c_eta;            /* sqrt(L) * eta, i.e. sqrt(2 L ln m) for eta = sqrt(2 ln m) */
  int32_t beam;           /* beam width W: nodes expanded per iteration, 1..ORC_MAX_BEAM */
} orc_params;

#define ORC_MAX_BEAM 8

enum { C_EXPANSIONS = 0, C_EDGES, C_VISITED_SKIP, C_A_REJECT, C_A_ACCEPT, C_H_TESTS, C_H_PASS,
       C_NDIST, C_INSERTS, C_STATUS, C_NCOUNTERS };

/* Outcome codes of one test: 0 reject by A >= 1, 1 accept by A <= 0, 2 H test, 3 degenerate accept,
 * 4 accept because R is not full (delta = infinity), 5 accept (always-pass / cut-only), */
typedef struct {
  float A, H, T;
  int pass;
  int kind;
} orc_edge_result;

/* Step (5): H(e) = w_reg H_1(e) + sqrt(L) w_res H_2(e), with
 * H_1 = sum_{i=1..L} sgn(e[i]) (x'_i . a^i_{|e[i]|}) (in order i = 1..L) and
 * H_2 = sgn(e[0]) (x' . b_{|e[0]|}), read from the projection table t of the normalised
 * query vector x' (t[0][j] = x' . b_j, t[i][j] = x'_i . a^i_j).  cr = sqrt(L) w_res. */
static float statistic_H(const int8_t* cd, const float* t, float wr, float cr, int L, int m) {
  float h1 = 0.0f;
  for (int i = 1; i <= L; ++i) {
    int c = cd[i];
    int j = (c > 0 ? c : -c) - 1;
    float tv = t[(size_t)i * m + j];
    h1 = h1 + ((c > 0) ? tv : -tv);
  }
  int c0 = cd[0];
  int j0 = (c0 > 0 ? c0 : -c0) - 1;
  float h2 = (c0 > 0) ? t[j0] : -t[j0];
  return wr * h1 + cr * h2;
}

/* The quantile lookup table of Sec. 4.3 (test_mode 3, frame Q): the variance of
 * N^{e,x}_min is bounded, 0 <= var <= L, so it is tabulated on 256 L bins of width 1/256;
 * the test uses the bin's upper edge, whose quantile A c + z sqrt(var) is slightly smaller
 * than the true one (z < 0), which keeps the guarantee. */
static float var_table_up(float var, int L) {
  int bin = (int)(var * 256.0f);
  if (bin < 0) bin = 0;
  if (bin > 256 * L - 1) bin = 256 * L - 1;
  return (float)(bin + 1) * (1.0f / 256.0f);
}

/* Step (4) and Eq. (LB): T_r(e) = F^{-1}_{e,eps}(A), the eps-quantile of
 * N(A sqrt(2 L ln m), w_reg^2 + L w_res^2 - L A^2 / (L + 1)) of Eq. (N_ex_min):
 * T = A c + z sqrt(var) with c = sqrt(2 L ln m) and z = Phi^{-1}(eps).  L w_res^2 = cr^2. */
static float threshold_T(float A, float wr, float cr, int L, const orc_params* P) {
  float Lf = (float)L;
  float var = (wr * wr + cr * cr) - (Lf * (A * A)) / (Lf + 1.0f);
  if (P->test_mode == 3) var = var_table_up(var, L);
  return A * P->c_eta + P->z_eps * sqrtf(fmaxf(var, 0.0f));
}

/* Frame T (the default): the expansion of v in coordinates translated by -v, so the
 * query vector is x = q - v and u's edge vector e = u - v is unchanged.
 *   tx     = projection table of x' = x / ||x|| (built by the caller from x, step 5)
 *   dv     = ||x||^2, the exact FP32 distance of v that the search holds
 *   delta2 = squared distance of R's furthest element, full = |R| == efs
 * With p' = p - v, the paper's A_r (Eq. A_r) becomes
 *   A = (||x||^2 + ||e||^2 - delta^2) / (2 ||x|| ||e||)    (use delta^2 - 2r = ||x||^2).
 * Then Algorithm 2: A >= 1 rejects, A <= 0 accepts, else pass iff H - T >= 0. */
static orc_edge_result edge_test_T(const float* tx, float dv, float delta2, int full, const int8_t* cd, float en,
                                   float wr, float cr, int L, int m, const orc_params* P) {
  orc_edge_result r = {0.0f, 0.0f, 0.0f, 1, 4};
  if (!full) return r;                       /* delta = infinity: every neighbour passes */
  if (P->test_mode == 2) { r.kind = 5; return r; }
  if (en == 0.0f || dv == 0.0f) { r.kind = 3; return r; }
  float xn = sqrtf(dv);
  float A = ((dv + en * en) - delta2) / (2.0f * (xn * en));
  r.A = A;
  if (A >= 1.0f) { r.pass = 0; r.kind = 0; return r; }
  if (A <= 0.0f) { r.pass = 1; r.kind = 1; return r; }
  if (P->test_mode == 1) { r.pass = 1; r.kind = 5; return r; }
  r.H = statistic_H(cd, tx, wr, cr, L, m);
  r.T = threshold_T(A, wr, cr, L, P);
  r.pass = (r.H - r.T) >= 0.0f;
  r.kind = 2;
  return r;
}

/* Frame Q, the paper-literal form: tq = table of q' = q / ||q||, A_r per Eq. (A_r) with
 * r = ||p||^2/2 - p.q; vq = v.q and un2 = ||u||^2 are plain FP32 dot products. */
static orc_edge_result edge_test_Q(const float* tq, float qn, float vq, float r_, float un2, int full,
                                   const int8_t* cd, float en, float wr, float cr, int L, int m,
                                   const orc_params* P) {
  orc_edge_result r = {0.0f, 0.0f, 0.0f, 1, 4};
  if (!full) return r;
  if (P->test_mode == 2) { r.kind = 5; return r; }
  if (en == 0.0f || qn == 0.0f) { r.kind = 3; return r; }
  float A = ((un2 / 2.0f - r_) - vq) / (qn * en);
  r.A = A;
  if (A >= 1.0f) { r.pass = 0; r.kind = 0; return r; }
  if (A <= 0.0f) { r.pass = 1; r.kind = 1; return r; }
  if (P->test_mode == 1) { r.pass = 1; r.kind = 5; return r; }
  r.H = statistic_H(cd, tq, wr, cr, L, m);
  r.T = threshold_T(A, wr, cr, L, P);
  r.pass = (r.H - r.T) >= 0.0f;
  r.kind = 2;
  return r;
}

/* The table of step (5) for a query vector y: y' = y / ||y|| coordinate by coordinate
 * (FP32 division), then orc_project(y').  `yn` = ||y|| > 0; `tmp` holds d floats. */
static void normalised_table(const float* y, float yn, int d, int L, int m, const float* A, const float* B,
                             float* tmp, float* t) {
  for (int k = 0; k < d; ++k) tmp[k] = y[k] / yn;
  orc_project(tmp, d, L, m, A, B, t);
}

/* ------------------------------------------------------------------------- */
/* SimHash test with the residual remedy (Sec. 3.1, Lemma 4.1)                */
/* ------------------------------------------------------------------------- */
/* K sign bits per edge: bit i of edge e = u - v is [S_i . e >= 0] (sgn(0) = +1), S_i the
 * K random vectors N(0, I_d); words of 64 bits, bit i in word i / 64 at position i % 64.
 * ||e|| is the plain sequential FP32 norm.  All dot products are sequential FP32 sums.
 * In the frame translated by -v the query vector is x = q - v, whose bits are
 * [S_i . x >= 0]. */
typedef struct {
  int K;                 /* hash bits, a multiple of 64, <= 192 */
  const float* S;        /* K x d */
  const uint64_t* bits;  /* [n*R][K/64] */
  const float* en;       /* [n*R] */
  const float* acrit;    /* [K+1]: pass iff A <= acrit[#Col] */
} orc_simhash;

int orc_simhash_build(const float* X, int64_t n, int d, const int32_t* nbrs, int R, int K, const float* S,
                      uint64_t* bits, float* en) {
  if (K < 64 || K % 64 != 0 || K > 192) return ORC_E_INVAL;
  const int W = K / 64;
  int fail = 0;
#pragma omp parallel
  {
    float* e = (float*)malloc(sizeof(float) * (size_t)d);
    if (!e) {
#pragma omp atomic write
      fail = 1;
    } else {
#pragma omp for schedule(dynamic, 64)
      for (int64_t v = 0; v < n; ++v) {
        const float* xv = X + (size_t)v * d;
        for (int s = 0; s < R; ++s) {
          size_t es = (size_t)v * R + s;
          int32_t u = nbrs[es];
          for (int w = 0; w < W; ++w) bits[es * W + w] = 0;
          en[es] = 0.0f;
          if (u < 0) continue;
          const float* xu = X + (size_t)u * d;
          for (int k = 0; k < d; ++k) e[k] = xu[k] - xv[k];
          en[es] = sqrtf(dot_f32(e, e, d));
          for (int i = 0; i < K; ++i)
            if (dot_f32(S + (size_t)i * d, e, d) >= 0.0f) bits[es * W + i / 64] |= (uint64_t)1 << (i % 64);
        }
      }
      free(e);
    }
  }
  return fail ? ORC_E_NOMEM : ORC_OK;
}

/* Thresholds of the test.  #Col ~ Binomial(K, 1 - theta/pi) for the angle theta between
 * e and x; u is closer than delta iff theta <= theta_max = arccos(A).  Hoeffding:
 * P(#Col <= K p - t) <= exp(-2 t^2 / K) = eps gives t = sqrt(K ln(1/eps) / 2), so the
 * test passes iff #Col >= K (1 - theta_max / pi) - t, i.e. iff
 * theta_max >= pi (1 - (#Col + t) / K), i.e. (cos decreasing) A <= cos(pi (1 - (#Col + t) / K));
 * acrit[c] is that cosine in FP64 rounded once to FP32, 1 when (c + t) / K >= 1. */
int orc_simhash_acrit(int K, double eps, float* acrit) {
  if (K < 1 || !(eps > 0.0 && eps < 1.0)) return ORC_E_INVAL;
  const double pi = 3.14159265358979323846;
  const double t = sqrt((double)K * log(1.0 / eps) / 2.0);
  for (int c = 0; c <= K; ++c) {
    const double r = ((double)c + t) / (double)K;
    acrit[c] = r >= 1.0 ? 1.0f : (float)cos(pi * (1.0 - r));
  }
  return ORC_OK;
}

static orc_edge_result edge_test_simhash(const orc_simhash* sh, size_t es, const uint64_t* bx, float dv, float xn,
                                         float delta2, int full, const orc_params* P) {
  orc_edge_result r = {0.0f, 0.0f, 0.0f, 1, 4};
  if (!full) return r;
  if (P->test_mode == 2) { r.kind = 5; return r; }
  const float en = sh->en[es];
  if (en == 0.0f || dv == 0.0f) { r.kind = 3; return r; }
  float A = ((dv + en * en) - delta2) / (2.0f * (xn * en));
  r.A = A;
  if (A >= 1.0f) { r.pass = 0; r.kind = 0; return r; }
  if (A <= 0.0f) { r.pass = 1; r.kind = 1; return r; }
  if (P->test_mode == 1) { r.pass = 1; r.kind = 5; return r; }
  const int W = sh->K / 64;
  int diff = 0;
  for (int w = 0; w < W; ++w) diff += __builtin_popcountll(sh->bits[es * W + w] ^ bx[w]);
  const int col = sh->K - diff;
  r.H = (float)col;
  r.T = sh->acrit[col];
  r.pass = A <= sh->acrit[col];
  r.kind = 2;
  return r;
}

/* ------------------------------------------------------------------------- */
/* Lazily built per-node index data (codes and weights)                       */
/* ------------------------------------------------------------------------- */
typedef struct {
  const float* X; int64_t n; int d;  /* the rows the search reads */
  const int32_t* nbrs; int R;
  int L, m;
  const float* A; const float* B;
  int8_t* codes; float* enorm; float* wreg; float* cres;
  uint8_t* ready; /* NULL: everything precomputed; else 0 = not built, 1 = building, 2 = built */
  const float* Xi; /* the FP32 rows of the index (codes, and the v of x = q - v) */
} orc_index;

static void ensure_node(const orc_index* ix, int64_t v, float* scratch) {
  if (!ix->ready) return;
  uint8_t st = __atomic_load_n(&ix->ready[v], __ATOMIC_ACQUIRE);
  if (st == 2) return;
  uint8_t expect = 0;
  if (__atomic_compare_exchange_n(&ix->ready[v], &expect, 1, 0, __ATOMIC_ACQ_REL, __ATOMIC_ACQUIRE)) {
    build_node(ix->Xi, ix->d, ix->nbrs, ix->R, ix->L, ix->m, ix->A, ix->B, v, ix->codes, ix->enorm, ix->wreg,
               ix->cres, scratch);
    __atomic_store_n(&ix->ready[v], 2, __ATOMIC_RELEASE);
  } else {
    while (__atomic_load_n(&ix->ready[v], __ATOMIC_ACQUIRE) != 2) { /* another thread is building v */ }
  }
}

/* ------------------------------------------------------------------------- */
/* Graph search, Algorithm 1                                                  */
/* ------------------------------------------------------------------------- */
/* Readings:
 *  - termination: R holds (dist, id, expanded); repeatedly expand the unexpanded
 *    entry of R with the smallest (dist, id); stop when none is left;
 *  - delta and |R| = efs are frozen at the start of an expansion for every test
 *    over v's edges; the exact distances of the neighbours that pass are then
 *    inserted in ascending (dist, id) order, each only if |R| < efs or dist < delta
 *    of the list as it stands (Algorithm 1's "dist(u,q) < delta");
 *  - a neighbour counts as visited only once its exact distance is computed, so a
 *    neighbour that fails the test can pass later from another node (Sec. 3.1);
 *  - beam width W: one iteration expands the W unexpanded entries of R with the
 *    smallest (dist, id) (fewer when fewer are left), all marked expanded at its start,
 *    with delta and |R| = efs frozen for the whole iteration; the nodes are taken in
 *    ascending (dist, id), each node's edges in slot order, a neighbour that passed
 *    earlier in the iteration counting as visited; the passes of the whole iteration are
 *    then inserted as above.  W = 1 is the pop-one loop of Algorithm 1.  The safety cap
 *    is checked before each iteration. */
typedef struct { float dist; int32_t id; int32_t expanded; } rentry;

static int rentry_less(float da, int32_t ia, float db, int32_t ib) {
  return (da < db) || (da == db && ia < ib);
}

static int cmp_cand(const void* a, const void* b) {
  const rentry* x = (const rentry*)a;
  const rentry* y = (const rentry*)b;
  if (rentry_less(x->dist, x->id, y->dist, y->id)) return -1;
  if (rentry_less(y->dist, y->id, x->dist, x->id)) return 1;
  return 0;
}

/* The exact visited set of one query: a byte per node, and the nodes touched so far
 * (so that resetting it costs what the query touched). */
typedef struct {
  uint8_t* seen;       /* n bytes */
  int32_t* touched; int64_t ntouched, cap_touched;
} visited_set;

static int vis_mark(visited_set* vs, int32_t id) {
  if (vs->seen[id]) return 1;
  vs->seen[id] = 1;
  if (vs->ntouched == vs->cap_touched) {
    int64_t nc = vs->cap_touched ? 2 * vs->cap_touched : 4096;
    int32_t* t = (int32_t*)realloc(vs->touched, sizeof(int32_t) * (size_t)nc);
    if (!t) return 0;
    vs->touched = t;
    vs->cap_touched = nc;
  }
  vs->touched[vs->ntouched++] = id;
  return 1;
}

static void vis_reset(visited_set* vs) {
  for (int64_t i = 0; i < vs->ntouched; ++i) vs->seen[vs->touched[i]] = 0;
  vs->ntouched = 0;
}

/* Insert c into sorted R (size *len, capacity ef) under Algorithm 1's rule. Returns 1 if inserted. */
static int r_insert(rentry* R, int* len, int ef, float dist, int32_t id) {
  if (*len == ef && !(dist < R[ef - 1].dist)) return 0;
  int pos = *len < ef ? *len : ef - 1;
  while (pos > 0 && rentry_less(dist, id, R[pos - 1].dist, R[pos - 1].id)) {
    R[pos] = R[pos - 1];
    --pos;
  }
  R[pos].dist = dist;
  R[pos].id = id;
  R[pos].expanded = 0;
  if (*len < ef) ++*len;
  return 1;
}

/* One query.  Scratch: tq / tx hold (L+1) m floats each, scratch 2 d floats. */
static int search_one(const orc_index* ix, const int32_t* nbrs_plain, int32_t entry, const float* q,
                      const int32_t* perm, const orc_simhash* sh, const orc_params* P, rentry* R, visited_set* vs,
                      rentry* cand, float* tq, float* tx, float* scratch, int64_t* cnt, int32_t* tr_v, float* tr_dv,
                      float* tr_d2, int* len_out) {
  const int d = ix->d, Rdeg = ix->R, L = ix->L, m = ix->m, ef = P->ef;
  const int peos = (P->routing == 1);
  const int simhash = (P->routing == 2);
  const int32_t* nbr = peos ? ix->nbrs : nbrs_plain;
  float* qi = scratch;     /* the query in the index's coordinates (permuted when perm is given) */
  float* xv = scratch + d; /* x = q - v of the expansion, then x' */
  float qn = 0.0f;
  uint64_t bx[3];   /* SimHash: the bits of x = q - v of the node being expanded */
  for (int t = 0; t < d; ++t) qi[t] = perm ? q[perm[t]] : q[t];
  if (peos && P->frame == 1) {
    /* frame Q: the table of q' = q / ||q||, built once per query (Algorithm 2) */
    qn = sqrtf(dot_f32(q, q, d));
    if (qn > 0.0f) normalised_table(qi, qn, d, L, m, ix->A, ix->B, xv, tq);
  }
  vis_reset(vs);
  int len = 0;
  *len_out = 0;
  float d0 = orc_dist2_f32(q, ix->X + (size_t)entry * d, d);
  cnt[C_NDIST]++;
  r_insert(R, &len, ef, d0, entry);
  if (!vis_mark(vs, entry)) return ORC_E_NOMEM;
  for (;;) {
    /* the W unexpanded entries with the smallest (dist, id): R is sorted by (dist, id) */
    int32_t bv[ORC_MAX_BEAM];
    float bd[ORC_MAX_BEAM];
    int nb = 0;
    for (int i = 0; i < len && nb < P->beam; ++i)
      if (!R[i].expanded) {
        R[i].expanded = 1;
        bv[nb] = R[i].id;
        bd[nb] = R[i].dist;
        ++nb;
      }
    if (nb == 0) break;
    if (cnt[C_EXPANSIONS] >= P->max_expansions) { cnt[C_STATUS] = ORC_E_OVERFLOW; break; }
    int full = (len == ef);
    float delta2 = full ? R[ef - 1].dist : INFINITY;
    int nc = 0;
    for (int b = 0; b < nb; ++b) {
      int32_t v = bv[b];
      float dv = bd[b];
      if (tr_v && cnt[C_EXPANSIONS] < P->trace_cap) {
        tr_v[cnt[C_EXPANSIONS]] = v;
        tr_dv[cnt[C_EXPANSIONS]] = dv;
        tr_d2[cnt[C_EXPANSIONS]] = delta2;
      }
      cnt[C_EXPANSIONS]++;
      float xn = sqrtf(dv);
      const float* vrow = ix->Xi + (size_t)v * d;  /* the index's (FP32, possibly permuted) row of v */
      if (simhash && full) {
        for (int k = 0; k < d; ++k) xv[k] = q[k] - ix->X[(size_t)v * d + k];
        for (int w = 0; w < sh->K / 64; ++w) bx[w] = 0;
        for (int i = 0; i < sh->K; ++i)
          if (dot_f32(sh->S + (size_t)i * d, xv, d) >= 0.0f) bx[i / 64] |= (uint64_t)1 << (i % 64);
      }
      float vq = 0.0f, r_ = 0.0f;
      if (peos) {
        ensure_node(ix, v, scratch + 2 * d);
        if (full && P->frame == 0 && P->test_mode == 0 && dv > 0.0f) {
          /* step (5) in the frame translated by -v: the table of x' = (q - v) / ||q - v|| */
          for (int k = 0; k < d; ++k) xv[k] = qi[k] - vrow[k];
          normalised_table(xv, xn, d, L, m, ix->A, ix->B, xv, tx);
        }
        if (full && P->frame == 1) {
          /* Eq. (A_r): v.q and r = ||p||^2 / 2 - p.q, p the efs-th entry of R */
          const float* xp = ix->X + (size_t)R[ef - 1].id * d;
          vq = dot_f32(ix->X + (size_t)v * d, q, d);
          r_ = dot_f32(xp, xp, d) / 2.0f - dot_f32(xp, q, d);
        }
      }
      for (int s = 0; s < Rdeg; ++s) {
        int32_t u = nbr[(size_t)v * Rdeg + s];
        if (u < 0) continue;
        cnt[C_EDGES]++;
        if (vs->seen[u]) { cnt[C_VISITED_SKIP]++; continue; }
        if (simhash) {
          orc_edge_result er = edge_test_simhash(sh, (size_t)v * Rdeg + s, bx, dv, xn, delta2, full, P);
          if (er.kind == 0) cnt[C_A_REJECT]++;
          if (er.kind == 1) cnt[C_A_ACCEPT]++;
          if (er.kind == 2) { cnt[C_H_TESTS]++; if (er.pass) cnt[C_H_PASS]++; }
          if (!er.pass) continue;
        }
        if (peos) {
          size_t es = (size_t)v * Rdeg + s;
          orc_edge_result er;
          if (P->frame == 0)
            er = edge_test_T(tx, dv, delta2, full, ix->codes + es * (L + 1), ix->enorm[es], ix->wreg[es], ix->cres[es],
                             L, m, P);
          else {
            const float* xu = ix->X + (size_t)u * d;
            er = edge_test_Q(tq, qn, vq, r_, dot_f32(xu, xu, d), full, ix->codes + es * (L + 1), ix->enorm[es],
                             ix->wreg[es], ix->cres[es], L, m, P);
          }
          if (er.kind == 0) cnt[C_A_REJECT]++;
          if (er.kind == 1) cnt[C_A_ACCEPT]++;
          if (er.kind == 2) { cnt[C_H_TESTS]++; if (er.pass) cnt[C_H_PASS]++; }
          if (!er.pass) continue;
        }
        if (!vis_mark(vs, u)) return ORC_E_NOMEM;
        cand[nc].dist = orc_dist2_f32(q, ix->X + (size_t)u * d, d);
        cand[nc].id = u;
        cand[nc].expanded = 0;
        cnt[C_NDIST]++;
        nc++;
      }
    }
    qsort(cand, (size_t)nc, sizeof(rentry), cmp_cand);
    for (int c = 0; c < nc; ++c) cnt[C_INSERTS] += r_insert(R, &len, ef, cand[c].dist, cand[c].id);
    *len_out = len;
  }
  *len_out = len;
  return ORC_OK;
}

/* Search nq queries.  Plain routing reads `nbrs` and needs no index data; PEOs reads
 * codes/enorm/wreg/cres (layouts as in orc_build_codes), built lazily per node when
 * `ready` is non-NULL, from the index rows Xi (NULL: X).
 * ids_out/dists_out: [nq][k] (id -1 / +inf when fewer than k results);
 * counters: [nq][C_NCOUNTERS] int64; trace arrays [nq][trace_cap] (may be NULL). */
int orc_search(const float* X, int64_t n, int d, const int32_t* nbrs, int R, int32_t entry,
               int8_t* codes, float* enorm, float* wreg, float* cres, uint8_t* ready,
               const float* A, const float* B, int L, int m,
               const float* Q, int64_t nq, const orc_params* P,
               int32_t* ids_out, float* dists_out, int64_t* counters,
               int32_t* tr_v, float* tr_dv, float* tr_d2, const float* Xr, const float* Xi,
               const int32_t* perm, const int32_t* entries, const orc_simhash* sh) {
  if (P->k <= 0 || P->ef < P->k || R <= 0 || entry < 0 || entry >= n) return ORC_E_INVAL;
  if (P->beam < 1 || P->beam > ORC_MAX_BEAM) return ORC_E_INVAL;
  if (P->routing == 2 && (!sh || sh->K < 64 || sh->K > 192 || sh->K % 64)) return ORC_E_INVAL;
  if (entries)
    for (int64_t qi = 0; qi < nq; ++qi)
      if (entries[qi] < 0 || entries[qi] >= n) return ORC_E_INVAL;
  if (P->routing == 1 && (d % L != 0 || !codes || !enorm || !wreg || !cres)) return ORC_E_INVAL;
  /* codes and the v of x = q - v come from the index's own vectors Xi (the FP32 rows),
   * which differ from X when the search reads a reduced-precision copy */
  orc_index ix = {X, n, d, nbrs, R, L, m, A, B, codes, enorm, wreg, cres, ready, Xi ? Xi : X};
  int fail = 0;
#pragma omp parallel
  {
    size_t tw = (size_t)(L + 1) * (size_t)m;
    rentry* Rl = (rentry*)malloc(sizeof(rentry) * (size_t)P->ef);
    rentry* cand = (rentry*)malloc(sizeof(rentry) * (size_t)R * (size_t)P->beam);
    float* tq = (float*)malloc(sizeof(float) * 2 * tw);
    float* scratch = (float*)malloc(sizeof(float) * (size_t)(4 * d + L + m));
    visited_set vs;
    memset(&vs, 0, sizeof(vs));
    vs.seen = (uint8_t*)calloc((size_t)n, 1);
    if (!Rl || !cand || !tq || !scratch || !vs.seen) {
#pragma omp atomic write
      fail = ORC_E_NOMEM;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t qi = 0; qi < nq; ++qi) {
        int64_t* cnt = counters + (size_t)qi * C_NCOUNTERS;
        memset(cnt, 0, sizeof(int64_t) * C_NCOUNTERS);
        int32_t* tv_ = tr_v ? tr_v + (size_t)qi * P->trace_cap : NULL;
        float* tdv_ = tr_dv ? tr_dv + (size_t)qi * P->trace_cap : NULL;
        float* td2_ = tr_d2 ? tr_d2 + (size_t)qi * P->trace_cap : NULL;
        int len = 0;
        int rc = search_one(&ix, nbrs, entries ? entries[qi] : entry, Q + (size_t)qi * d, perm, sh, P, Rl, &vs,
                            cand, tq, tq + tw, scratch, cnt, tv_, tdv_, td2_, &len);
        if (rc != ORC_OK) {
#pragma omp atomic write
          fail = rc;
        }
        if (Xr) {
          /* re-rank: exact FP32 distances of every entry of R from the full-precision
           * base, then R sorted again by (dist, id) */
          const float* q = Q + (size_t)qi * d;
          for (int j = 0; j < len; ++j) Rl[j].dist = orc_dist2_f32(q, Xr + (size_t)Rl[j].id * d, d);
          qsort(Rl, (size_t)len, sizeof(rentry), cmp_cand);
        }
        for (int j = 0; j < P->k; ++j) {
          ids_out[(size_t)qi * P->k + j] = j < len ? Rl[j].id : -1;
          dists_out[(size_t)qi * P->k + j] = j < len ? Rl[j].dist : INFINITY;
        }
      }
    }
    free(Rl); free(cand); free(tq); free(scratch);
    free(vs.seen); free(vs.touched);
  }
  return fail;
}

/* One PEOs test outside a search, for element-wise comparison of the test
 * statistics: query q, expanded node v with stored distance dv, list bound
 * delta2 (full list).  Frame T, or frame Q (P->frame = 1; p = the row of the list's
 * efs-th entry, the rest as in the search).  X are the rows the search reads, Xi the
 * index's (FP32, in the codes' coordinates when perm is given).  Outputs per out-edge
 * s of v: A, H, T, pass, kind. */
int orc_edge_stats(const float* X, const float* Xi, int64_t n, int d, const int32_t* nbrs, int R, int L, int m,
                   const float* A, const float* B, const int8_t* codes, const float* enorm, const float* wreg,
                   const float* cres, const float* q, const int32_t* perm, int32_t v, float dv,
                   float delta2, int32_t p, const orc_params* P,
                   float* A_out, float* H_out, float* T_out, int32_t* pass_out, int32_t* kind_out) {
  if (v < 0 || v >= n || (P->frame == 1 && (p < 0 || p >= n))) return ORC_E_INVAL;
  size_t tw = (size_t)(L + 1) * m;
  float* tq = (float*)malloc(sizeof(float) * (tw + 2 * (size_t)d));
  if (!tq) return ORC_E_NOMEM;
  float* qi = tq + tw;
  float* xv = qi + d;
  for (int t = 0; t < d; ++t) qi[t] = perm ? q[perm[t]] : q[t];
  memset(tq, 0, sizeof(float) * tw);
  float xn = sqrtf(dv);
  float qn = 0.0f, vq = 0.0f, r_ = 0.0f;
  if (P->frame == 1) {
    qn = sqrtf(dot_f32(q, q, d));
    if (qn > 0.0f) normalised_table(qi, qn, d, L, m, A, B, xv, tq);
    const float* xp = X + (size_t)p * d;
    vq = dot_f32(X + (size_t)v * d, q, d);
    r_ = dot_f32(xp, xp, d) / 2.0f - dot_f32(xp, q, d);
  } else if (dv > 0.0f) {
    for (int k = 0; k < d; ++k) xv[k] = qi[k] - Xi[(size_t)v * d + k];
    normalised_table(xv, xn, d, L, m, A, B, xv, tq);
  }
  for (int s = 0; s < R; ++s) {
    size_t es = (size_t)v * R + s;
    orc_edge_result er;
    if (P->frame == 1) {
      int32_t u = nbrs[es];
      float un2 = u >= 0 ? dot_f32(X + (size_t)u * d, X + (size_t)u * d, d) : 0.0f;
      er = edge_test_Q(tq, qn, vq, r_, un2, 1, codes + es * (L + 1), enorm[es], wreg[es], cres[es], L, m, P);
    } else {
      er = edge_test_T(tq, dv, delta2, 1, codes + es * (L + 1), enorm[es], wreg[es], cres[es], L, m, P);
    }
    A_out[s] = er.A; H_out[s] = er.H; T_out[s] = er.T; pass_out[s] = er.pass; kind_out[s] = er.kind;
  }
  free(tq);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Brute-force K-NN in FP64                                                   */
/* ------------------------------------------------------------------------- */
typedef struct { double dist; int32_t id; } dpair;

static int cmp_dpair(const void* a, const void* b) {
  const dpair* x = (const dpair*)a;
  const dpair* y = (const dpair*)b;
  if (x->dist < y->dist) return -1;
  if (x->dist > y->dist) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

/* Keep the k smallest (dist, id) of a stream in a sorted array (insertion). */
static void topk_push(dpair* top, int* len, int k, double dist, int32_t id) {
  if (*len == k) {
    dpair w = top[k - 1];
    if (!(dist < w.dist || (dist == w.dist && id < w.id))) return;
  }
  int pos = *len < k ? *len : k - 1;
  while (pos > 0 && (dist < top[pos - 1].dist || (dist == top[pos - 1].dist && id < top[pos - 1].id))) {
    top[pos] = top[pos - 1];
    --pos;
  }
  top[pos].dist = dist;
  top[pos].id = id;
  if (*len < k) ++*len;
}

int orc_knn_f64(const float* X, int64_t n, int d, const float* Q, int64_t nq, int k, int32_t* ids, double* dists) {
  if (k <= 0) return ORC_E_INVAL;
  int fail = 0;
#pragma omp parallel
  {
    dpair* top = (dpair*)malloc(sizeof(dpair) * (size_t)k);
    if (!top) {
#pragma omp atomic write
      fail = ORC_E_NOMEM;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t qi = 0; qi < nq; ++qi) {
        int len = 0;
        for (int64_t x = 0; x < n; ++x)
          topk_push(top, &len, k, dist2_f64(Q + (size_t)qi * d, X + (size_t)x * d, d), (int32_t)x);
        for (int j = 0; j < k; ++j) {
          ids[(size_t)qi * k + j] = j < len ? top[j].id : -1;
          dists[(size_t)qi * k + j] = j < len ? top[j].dist : INFINITY;
        }
      }
      free(top);
    }
  }
  return fail;
}

/* ------------------------------------------------------------------------- */
/* Graph builder: exact kNN + relative-neighbourhood pruning (FP64)           */
/* ------------------------------------------------------------------------- */
/* Relative-neighbourhood pruning of a candidate list sorted by (dist to x, id):
 * keep c unless an already kept s has d(s, c) < d(x, c); stop at R kept. */
static int rng_prune(const float* X, int d, const dpair* cand, int nc, int R, int32_t* out) {
  int kept = 0;
  for (int c = 0; c < nc && kept < R; ++c) {
    int ok = 1;
    for (int s = 0; s < kept; ++s) {
      if (dist2_f64(X + (size_t)out[s] * d, X + (size_t)cand[c].id * d, d) < cand[c].dist) { ok = 0; break; }
    }
    if (ok) out[kept++] = cand[c].id;
  }
  return kept;
}

/* ------------------------------------------------------------------------- */
/* Hierarchical entry: greedy descent through upper layers (HNSW-style)      */
/* ------------------------------------------------------------------------- */
/* One layer of the descent for every query.  The layer is a graph over n_l of the
 * base's nodes: ids[i] = the base row of local node i, nbrs[i*R + s] = local ids (-1
 * empty).  cur[qi] (in/out) is the query's local node.  Greedy search with a list of
 * one, as in an HNSW upper layer: from the current node c, the neighbour with the
 * smallest (dist, base id) is taken if its distance is strictly smaller than c's;
 * repeated until no neighbour is closer.  Distances are orc_dist2_f32. */
int orc_greedy_layer(const float* X, int d, const float* Q, int64_t nq, int64_t n_l, int R, const int32_t* ids,
                     const int32_t* nbrs, int32_t* cur, int64_t* hops) {
  for (int64_t qi = 0; qi < nq; ++qi)
    if (cur[qi] < 0 || cur[qi] >= n_l) return ORC_E_INVAL;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t qi = 0; qi < nq; ++qi) {
    const float* q = Q + (size_t)qi * d;
    int32_t c = cur[qi];
    float dc = orc_dist2_f32(q, X + (size_t)ids[c] * d, d);
    int64_t h = 0;
    for (;;) {
      int32_t best = -1;
      float db = 0.0f;
      for (int s = 0; s < R; ++s) {
        int32_t u = nbrs[(size_t)c * R + s];
        if (u < 0 || u >= n_l) continue;
        float du = orc_dist2_f32(q, X + (size_t)ids[u] * d, d);
        if (best < 0 || du < db || (du == db && ids[u] < ids[best])) {
          best = u;
          db = du;
        }
      }
      if (best < 0 || !(db < dc)) break;
      c = best;
      dc = db;
      ++h;
    }
    cur[qi] = c;
    if (hops) hops[qi] = h;
  }
  return ORC_OK;
}

static int64_t bfs_reach(const int32_t* nbrs, int64_t n, int R, int32_t entry, uint8_t* seen, int32_t* queue) {
  memset(seen, 0, (size_t)n);
  int64_t head = 0, tail = 0;
  seen[entry] = 1;
  queue[tail++] = entry;
  while (head < tail) {
    int32_t x = queue[head++];
    for (int s = 0; s < R; ++s) {
      int32_t y = nbrs[(size_t)x * R + s];
      if (y >= 0 && !seen[y]) { seen[y] = 1; queue[tail++] = y; }
    }
  }
  return tail;
}

/* Steps: (1) Kc exact nearest candidates per node (FP64, ties by id); (2) prune
 * to <= R; (3) add reverse edges: a node's list becomes the union of its own and
 * offered edges, ordered by (dist, id) and cut to its ucap nearest, re-pruned
 * with the same rule when longer than R; (4) entry = the node
 * nearest the centroid; (5) while some node is unreachable from the entry, give
 * the smallest-id unreachable node z an in-edge from its nearest reachable node
 * with a free slot (or, if none has one, replace that node's furthest edge). */
int orc_build_graph(const float* X, int64_t n, int d, int R, int Kc, int ucap, int32_t* nbrs, int32_t* entry_out) {
  if (n < 2 || R <= 0 || Kc < R || ucap < R) return ORC_E_INVAL;
  if (Kc > n - 1) Kc = (int)(n - 1);
  int32_t* fwd = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * R);
  int32_t* fdeg = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  if (!fwd || !fdeg) { free(fwd); free(fdeg); return ORC_E_NOMEM; }
  int fail = 0;
#pragma omp parallel
  {
    dpair* top = (dpair*)malloc(sizeof(dpair) * (size_t)Kc);
    if (!top) {
#pragma omp atomic write
      fail = ORC_E_NOMEM;
    } else {
#pragma omp for schedule(dynamic, 16)
      for (int64_t x = 0; x < n; ++x) {
        int len = 0;
        for (int64_t y = 0; y < n; ++y) {
          if (y == x) continue;
          topk_push(top, &len, Kc, dist2_f64(X + (size_t)x * d, X + (size_t)y * d, d), (int32_t)y);
        }
        fdeg[x] = rng_prune(X, d, top, len, R, fwd + (size_t)x * R);
      }
      free(top);
    }
  }
  if (fail) { free(fwd); free(fdeg); return fail; }
  /* reverse edges */
  int32_t* rdeg = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  int64_t* roff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!rdeg || !roff) { free(fwd); free(fdeg); free(rdeg); free(roff); return ORC_E_NOMEM; }
  for (int64_t x = 0; x < n; ++x)
    for (int s = 0; s < fdeg[x]; ++s) rdeg[fwd[(size_t)x * R + s]]++;
  roff[0] = 0;
  for (int64_t y = 0; y < n; ++y) roff[y + 1] = roff[y] + rdeg[y];
  int32_t* rev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(roff[n] > 0 ? roff[n] : 1));
  int32_t* rfill = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  if (!rev || !rfill) { free(fwd); free(fdeg); free(rdeg); free(roff); free(rev); free(rfill); return ORC_E_NOMEM; }
  for (int64_t x = 0; x < n; ++x)
    for (int s = 0; s < fdeg[x]; ++s) {
      int32_t y = fwd[(size_t)x * R + s];
      rev[roff[y] + rfill[y]++] = (int32_t)x;
    }
  int32_t* deg = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  if (!deg) { fail = ORC_E_NOMEM; }
#pragma omp parallel
  {
    int64_t maxu = 0;
    for (int64_t y = 0; y < n; ++y) if (fdeg[y] + rdeg[y] > maxu) maxu = fdeg[y] + rdeg[y];
    dpair* uni = (dpair*)malloc(sizeof(dpair) * (size_t)(maxu > 0 ? maxu : 1));
    if (!uni || fail) {
#pragma omp atomic write
      fail = ORC_E_NOMEM;
    } else {
#pragma omp for schedule(dynamic, 64)
      for (int64_t y = 0; y < n; ++y) {
        int nu = 0;
        for (int s = 0; s < fdeg[y]; ++s) { uni[nu].id = fwd[(size_t)y * R + s]; nu++; }
        for (int64_t t = roff[y]; t < roff[y + 1]; ++t) {
          int32_t x = rev[t];
          int dup = 0;
          for (int w = 0; w < nu; ++w) if (uni[w].id == x) { dup = 1; break; }
          if (!dup) { uni[nu].id = x; nu++; }
        }
        for (int w = 0; w < nu; ++w) uni[w].dist = dist2_f64(X + (size_t)y * d, X + (size_t)uni[w].id * d, d);
        qsort(uni, (size_t)nu, sizeof(dpair), cmp_dpair);
        if (nu > ucap) nu = ucap;
        int32_t* out = nbrs + (size_t)y * R;
        if (nu <= R) {
          for (int w = 0; w < nu; ++w) out[w] = uni[w].id;
          deg[y] = nu;
        } else {
          deg[y] = rng_prune(X, d, uni, nu, R, out);
        }
        for (int w = deg[y]; w < R; ++w) out[w] = -1;
      }
    }
    free(uni);
  }
  free(fwd); free(fdeg); free(rdeg); free(roff); free(rev); free(rfill);
  if (fail) { free(deg); return fail; }
  /* entry: nearest node to the centroid */
  double* cen = (double*)calloc((size_t)d, sizeof(double));
  uint8_t* seen = (uint8_t*)malloc((size_t)n);
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!cen || !seen || !queue) { free(deg); free(cen); free(seen); free(queue); return ORC_E_NOMEM; }
  for (int64_t x = 0; x < n; ++x)
    for (int k = 0; k < d; ++k) cen[k] += (double)X[(size_t)x * d + k];
  for (int k = 0; k < d; ++k) cen[k] /= (double)n;
  int32_t entry = 0;
  double best = INFINITY;
  for (int64_t x = 0; x < n; ++x) {
    double acc = 0.0;
    for (int k = 0; k < d; ++k) { double t = (double)X[(size_t)x * d + k] - cen[k]; acc += t * t; }
    if (acc < best) { best = acc; entry = (int32_t)x; }
  }
  /* connectivity repair */
  int64_t reached = bfs_reach(nbrs, n, R, entry, seen, queue);
  while (reached < n) {
    int32_t z = 0;
    while (seen[z]) ++z;
    int32_t wbest = -1, wfull = -1;
    double dbest = INFINITY, dfull = INFINITY;
    for (int64_t w = 0; w < n; ++w) {
      if (!seen[w]) continue;
      double dd = dist2_f64(X + (size_t)w * d, X + (size_t)z * d, d);
      if (deg[w] < R) { if (dd < dbest) { dbest = dd; wbest = (int32_t)w; } }
      else if (dd < dfull) { dfull = dd; wfull = (int32_t)w; }
    }
    int32_t w = wbest >= 0 ? wbest : wfull;
    double dz = wbest >= 0 ? dbest : dfull;
    int32_t* out = nbrs + (size_t)w * R;
    int len = deg[w] < R ? deg[w] : R - 1; /* a full list drops its furthest edge */
    int pos = len;
    while (pos > 0) {
      double dp = dist2_f64(X + (size_t)w * d, X + (size_t)out[pos - 1] * d, d);
      if (dz < dp || (dz == dp && z < out[pos - 1])) { out[pos] = out[pos - 1]; --pos; } else break;
    }
    out[pos] = z;
    deg[w] = len + 1;
    reached = bfs_reach(nbrs, n, R, entry, seen, queue);
  }
  *entry_out = entry;
  free(deg); free(cen); free(seen); free(queue);
  return ORC_OK;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}
