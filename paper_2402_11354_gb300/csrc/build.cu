// Index-time PEOs data (Sec. 4.2 steps (1)-(3)): per edge e = u - v the block
// norms, ||e||, w_reg, e_res and the L+1 extreme-value codes, and the edge's node
// term of the statistic (S(t(v)), from v's projection table); per node the
// projection table.  One CTA per node; all of a node's edges (R <= 64) are staged
// in shared memory.  With a dimension permutation (Appendix D.1) both work on the
// permuted vectors: coordinate k of a row is read from coordinate perm[k].  Every sum
// is a plain sequential FP32 sum (compiled with --fmad=false), one thread per output,
// so the results are reproducible bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "device.cuh"
#include "internal.h"

namespace peos {
namespace {

constexpr int kBuildThreads = 256;

__global__ void __launch_bounds__(kBuildThreads) build_codes_kernel(const float* __restrict__ X, long long n, int d,
                                                                    const int32_t* __restrict__ nbrs, int R, int L,
                                                                    int m, const float* __restrict__ A,
                                                                    const float* __restrict__ B,
                                                                    const int32_t* __restrict__ perm,
                                                                    const float* __restrict__ node_proj,
                                                                    int proj_stride, uint8_t* __restrict__ rec,
                                                                    size_t rec_stride, int bits, int cpw,
                                                                    int nwords) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int dp = d / L;
  float* e = reinterpret_cast<float*>(smem_raw);   // [R][d]  e, later e_res
  float* n2 = e + (size_t)R * d;                    // [R][L]  block norms squared
  float* bn = n2 + R * L;                           // [R][L]  block norms
  float* en = bn + R * L;                           // [R]
  float* wr = en + R;                               // [R]
  float* mean = wr + R;                             // [R]
  float* cr = mean + R;                             // [R]  sqrt(L) w_res
  float* proj = cr + R;                             // [R][L+1][m]
  int32_t* ids = reinterpret_cast<int32_t*>(proj + (size_t)R * (L + 1) * m);  // [R]
  int32_t* sel = ids + R;                                                      // [R][L+1] argmax j | sign << 16
  float* tvs = reinterpret_cast<float*>(sel + (size_t)R * (L + 1));           // [(L+1) m] t(v)
  const int tid = threadIdx.x;

  for (long long v = blockIdx.x; v < n; v += gridDim.x) {
    for (int s = tid; s < R; s += blockDim.x) ids[s] = nbrs[(size_t)v * R + s];
    for (int t = tid; t < (L + 1) * m; t += blockDim.x) tvs[t] = node_proj[(size_t)v * proj_stride + t];
    __syncthreads();
    for (int idx = tid; idx < R * d; idx += blockDim.x) {
      const int s = idx / d, k = idx - s * d;
      const int32_t u = ids[s];
      const int kk = perm ? __ldg(perm + k) : k;
      e[idx] = (u >= 0) ? (X[(size_t)u * d + kk] - X[(size_t)v * d + kk]) : 0.0f;
    }
    __syncthreads();
    // step (1): block norms
    for (int t = tid; t < R * L; t += blockDim.x) {
      const int s = t / L, i = t - s * L;
      const float* ei = e + (size_t)s * d + i * dp;
      float acc = 0.0f;
      for (int k = 0; k < dp; ++k) {
        const float x = ei[k];
        acc = acc + x * x;
      }
      n2[t] = acc;
      bn[t] = sqrtf(acc);
    }
    __syncthreads();
    for (int s = tid; s < R; s += blockDim.x) {
      float tot2 = 0.0f, sum = 0.0f;
      for (int i = 0; i < L; ++i) {
        tot2 = tot2 + n2[s * L + i];
        sum = sum + bn[s * L + i];
      }
      const float norm = sqrtf(tot2);
      en[s] = norm;
      if (norm == 0.0f) {
        wr[s] = 1.0f;
        cr[s] = 0.0f;
        mean[s] = 0.0f;
      } else {
        float w = sum / (sqrtf((float)L) * norm);
        if (w > 1.0f) w = 1.0f;
        wr[s] = w;
        cr[s] = sqrtf((float)L) * sqrtf(fmaxf(0.0f, 1.0f - w * w));
        mean[s] = sum / (float)L;
      }
    }
    __syncthreads();
    // step (3), i = 1..L: projections of e_i onto the a^i_j
    for (int t = tid; t < R * L * m; t += blockDim.x) {
      const int s = t / (L * m);
      const int rem = t - s * L * m;
      const int i = rem / m, j = rem - i * m;
      const float* a = A + ((size_t)i * m + j) * dp;
      const float* ei = e + (size_t)s * d + i * dp;
      float acc = 0.0f;
      for (int k = 0; k < dp; ++k) acc = acc + __ldg(a + k) * ei[k];
      proj[((size_t)s * (L + 1) + i + 1) * m + j] = acc;
    }
    __syncthreads();
    // step (1): e_res = e - e_reg, block i scaled by 1 - mean(||e_k||) / ||e_i||
    for (int idx = tid; idx < R * d; idx += blockDim.x) {
      const int s = idx / d, k = idx - s * d;
      const int i = k / dp;
      const float b = bn[s * L + i];
      const float coef = (b > 0.0f) ? (1.0f - mean[s] / b) : 0.0f;
      e[idx] = e[idx] * coef;
    }
    __syncthreads();
    // step (3), e[0]: projections of e_res onto the b_j
    for (int t = tid; t < R * m; t += blockDim.x) {
      const int s = t / m, j = t - s * m;
      const float* b = B + (size_t)j * d;
      const float* er = e + (size_t)s * d;
      float acc = 0.0f;
      for (int k = 0; k < d; ++k) acc = acc + __ldg(b + k) * er[k];
      proj[((size_t)s * (L + 1)) * m + j] = acc;
    }
    __syncthreads();
    // argmax_j |.|, lowest j on ties, sgn(0) = +1 (a degenerate edge, ||e|| = 0, gets +1)
    for (int t = tid; t < R * (L + 1); t += blockDim.x) {
      const int s = t / (L + 1);
      const float* p = proj + (size_t)t * m;
      int best = 0;
      float bv = fabsf(p[0]);
      for (int j = 1; j < m; ++j) {
        const float av = fabsf(p[j]);
        if (av > bv) {
          bv = av;
          best = j;
        }
      }
      const int neg = (en[s] != 0.0f && !(p[best] >= 0.0f)) ? 1 : 0;
      sel[t] = (en[s] == 0.0f ? 0 : best) | (neg << 16);
    }
    __syncthreads();
    // packed per edge (see code_bits)
    uint8_t* r = rec + (size_t)v * rec_stride;
    uint64_t* cwords = reinterpret_cast<uint64_t*>(r + rec_codes_offset(R));
    for (int t = tid; t < R * nwords; t += blockDim.x) {
      const int s = t / nwords, w = t - s * nwords;
      uint64_t word = 0;
      if (ids[s] >= 0) {
        for (int k = 0; k < cpw; ++k) {
          const int c = w * cpw + k;
          if (c > L) break;
          const int q = sel[s * (L + 1) + c];
          const uint64_t code = (uint64_t)(q & 0xffff) | ((uint64_t)(q >> 16) << (bits - 1));
          word |= code << (k * bits);
        }
      }
      cwords[(size_t)w * R + s] = word;
    }
    // node term S(t(v)) = w_reg sum_{c=1..L} sgn t(v)[c][j_c] + sqrt(L) w_res sgn t(v)[0][j_0]
    for (int s = tid; s < R; s += blockDim.x) {
      const bool ok = ids[s] >= 0;
      float svv = 0.0f;
      if (ok) {
        float h1 = 0.0f;
        for (int c = 1; c <= L; ++c) {
          const int q = sel[s * (L + 1) + c];
          const float val = tvs[c * m + (q & 0xffff)];
          h1 = h1 + ((q >> 16) ? -val : val);
        }
        const int q0 = sel[s * (L + 1)];
        const float v0 = tvs[q0 & 0xffff];
        const float h2 = (q0 >> 16) ? -v0 : v0;
        svv = wr[s] * h1 + cr[s] * h2;
      }
      reinterpret_cast<float4*>(r)[s] = ok ? make_float4(en[s], wr[s], cr[s], svv) : make_float4(0.f, 0.f, 0.f, 0.f);
      reinterpret_cast<int32_t*>(r + rec_ids_offset(R))[s] = ids[s];
    }
    // zero the gap before the codes and the padding after them
    for (size_t b = rec_ids_offset(R) + 4 * (size_t)R + tid; b < rec_codes_offset(R); b += blockDim.x) r[b] = 0;
    const size_t used = rec_codes_offset(R) + 8 * (size_t)nwords * R;
    for (size_t b = used + tid; b < rec_stride; b += blockDim.x) r[b] = 0;
    __syncthreads();
  }
}

// projection table of every node: out[v][c][j], one thread per entry
__global__ void node_proj_kernel(const float* __restrict__ X, long long n, int d, int L, int m,
                                 const float* __restrict__ A, const float* __restrict__ B,
                                 const int32_t* __restrict__ perm, float* __restrict__ out, int out_stride) {
  const int tw = out_stride;  // (L+1)*m entries, then zero padding
  const int dp = d / L;
  const long long total = n * (long long)tw;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long v = t / tw;
    const int e = (int)(t - v * tw);
    const int c = e / m, j = e - c * m;
    const float* x = X + (size_t)v * d;
    float acc = 0.0f;
    if (c > L) {
      // padding entry
    } else if (c == 0) {
      // block by block: a sequential partial sum per block of d/L dims, then the partials
      const float* b = B + (size_t)j * d;
      for (int i = 0; i < L; ++i) {
        float part = 0.0f;
        for (int k = 0; k < dp; ++k) {
          const int t = i * dp + k;
          part = part + __ldg(b + t) * __ldg(x + (perm ? __ldg(perm + t) : t));
        }
        acc = acc + part;
      }
    } else {
      const int i = c - 1;
      const float* a = A + ((size_t)i * m + j) * dp;
      for (int k = 0; k < dp; ++k) {
        const int t = i * dp + k;
        acc = acc + __ldg(a + k) * __ldg(x + (perm ? __ldg(perm + t) : t));
      }
    }
    out[t] = acc;
  }
}

// ||v||^2 of every row, a plain sequential FP32 sum per row (one thread per row)
__global__ void row_norms_kernel(const float* __restrict__ X, long long n, int d, float* __restrict__ norms) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const float* x = X + (size_t)v * d;
    float acc = 0.0f;
    for (int k = 0; k < d; ++k) acc = acc + __ldg(x + k) * __ldg(x + k);
    norms[v] = acc;
  }
}

int num_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

// The compact index (8- or 16-bit edge scalars; Sec. 4.3's space analysis, Sec. 6.4's
// PEOs (Compact)): one warp per node rewrites its FP32 record.  Per scalar kind (||e||,
// w_reg, sqrt(L) w_res) over the node's valid edges: s = max |x|, step = s / Qb
// (Qb = 2^(bits-1) - 1), q = rint(x / step) clamped to [-Qb, Qb] (0 when step = 0); the
// search reads x' = (float) q * step.  The node term is recomputed from the stored
// weights, sv = w_reg' sum_{c=1..L} sgn t(v)[c][j_c] + (sqrt(L) w_res)' sgn t(v)[0][j_0]
// (the same FP32 order as build_codes_kernel), and kept in FP32, so that the statistic
// the search forms, (S(t(q)) - sv) / ||x||, is the one of the stored weights.  Ids and
// codes are copied unchanged.
template <int SB>
__global__ void compact_records_kernel(const uint8_t* __restrict__ src, size_t src_stride, long long n, int R,
                                       int words, const float* __restrict__ node_proj, int proj_stride, int L, int m,
                                       uint8_t* __restrict__ dst, size_t dst_stride) {
  using Q4 = typename std::conditional<SB == 16, short4, char4>::type;
  constexpr float kQb = SB == 16 ? 32767.0f : 127.0f;
  const int lane = threadIdx.x & 31;
  const int bits = code_bits(m), cpw = codes_per_word(m);
  const unsigned long long mask = (1ull << bits) - 1ull;
  const int half = 1 << (bits - 1);
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long v = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += warps) {
    const uint8_t* r = src + (size_t)v * src_stride;
    uint8_t* o = dst + (size_t)v * dst_stride;
    const float4* sc = reinterpret_cast<const float4*>(r);
    const int32_t* ids = reinterpret_cast<const int32_t*>(r + rec_ids_offset(R));
    const uint64_t* cs = reinterpret_cast<const uint64_t*>(r + rec_codes_offset(R));
    const float* tv = node_proj + (size_t)v * proj_stride;
    float4 x[2];
    int32_t id[2];
    float mx[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int sl = h * 32 + lane;
      id[h] = sl < R ? ids[sl] : -1;
      x[h] = sl < R ? sc[sl] : make_float4(0.f, 0.f, 0.f, 0.f);
      if (id[h] >= 0) {
        mx[0] = fmaxf(mx[0], fabsf(x[h].x));
        mx[1] = fmaxf(mx[1], fabsf(x[h].y));
        mx[2] = fmaxf(mx[2], fabsf(x[h].z));
      }
    }
    float step[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) mx[k] = fmaxf(mx[k], __shfl_xor_sync(kFull, mx[k], off));
      step[k] = mx[k] / kQb;
    }
    if (lane == 0) *reinterpret_cast<float4*>(o) = make_float4(step[0], step[1], step[2], 0.0f);
    auto quant = [&](float val, float st, bool ok) -> int {
      if (!ok || !(st > 0.0f)) return 0;
      float q = rintf(val / st);
      q = fminf(fmaxf(q, -kQb), kQb);
      return (int)q;
    };
    // 16-bit form: sv[R] then q[R]; 8-bit form: {q, sv} pairs of 8 bytes
    float* svo = reinterpret_cast<float*>(o + (SB == 16 ? rec_sv_offset(R) : rec_pair_offset() + 4));
    Q4* qo = reinterpret_cast<Q4*>(o + (SB == 16 ? rec_q_offset(R) : rec_pair_offset()));
    constexpr int kStep = SB == 16 ? 1 : 2;  // elements of 4 bytes (sv) / of sizeof(Q4) (q) per edge
    int32_t* io = reinterpret_cast<int32_t*>(o + rec_ids_offset(R, SB));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int sl = h * 32 + lane;
      if (sl < R) {
        const bool ok = id[h] >= 0;
        Q4 q;
        q.x = quant(x[h].x, step[0], ok);
        q.y = quant(x[h].y, step[1], ok);
        q.z = quant(x[h].z, step[2], ok);
        q.w = 0;
        float svv = 0.0f;
        if (ok) {
          const float wq = (float)q.y * step[1], cq = (float)q.z * step[2];
          // the edge's codes e[0..L] from its packed words: code c sits in word c / cpw
          float h1 = 0.0f, h2 = 0.0f;
          for (int c = 0; c <= L; ++c) {
            const unsigned long long word = cs[(size_t)(c / cpw) * R + sl];
            const int code = (int)((word >> ((c % cpw) * bits)) & mask);
            const float val = tv[c * m + (code & (half - 1))];
            const float sv_c = (code & half) ? -val : val;
            if (c == 0) h2 = sv_c; else h1 = h1 + sv_c;
          }
          svv = wq * h1 + cq * h2;
        }
        qo[(size_t)kStep * sl] = q;
        svo[(size_t)kStep * sl] = svv;
        io[sl] = id[h];
      }
    }
    // codes, then zero the gaps and the padding
    uint64_t* cd = reinterpret_cast<uint64_t*>(o + rec_codes_offset(R, SB));
    for (int t = lane; t < words * R; t += 32) cd[t] = cs[t];
    if (SB == 16)
      for (size_t b = rec_sv_offset(R) + 4 * (size_t)R + lane; b < rec_q_offset(R); b += 32) o[b] = 0;
    for (size_t b = rec_ids_offset(R, SB) + 4 * (size_t)R + lane; b < rec_codes_offset(R, SB); b += 32) o[b] = 0;
    for (size_t b = rec_codes_offset(R, SB) + 8 * (size_t)words * R + lane; b < dst_stride; b += 32) o[b] = 0;
  }
}

}  // namespace

cudaError_t launch_compact_records(const uint8_t* src, size_t src_stride, int64_t n, int R, int words,
                                   const float* node_proj, int proj_stride, int L, int m, int sbits, uint8_t* dst,
                                   size_t dst_stride, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (R > 64 || !node_proj) return cudaErrorInvalidValue;
  const int threads = 256;
  long long blocks = (n + 7) / 8;
  if (blocks > 65535LL * 16) blocks = 65535LL * 16;
  if (sbits == 16)
    compact_records_kernel<16><<<(unsigned)blocks, threads, 0, st>>>(src, src_stride, n, R, words, node_proj,
                                                                     proj_stride, L, m, dst, dst_stride);
  else if (sbits == 8)
    compact_records_kernel<8><<<(unsigned)blocks, threads, 0, st>>>(src, src_stride, n, R, words, node_proj,
                                                                    proj_stride, L, m, dst, dst_stride);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_build_codes(const float* X, int64_t n, int d, const int32_t* nbrs, int R, int L, int m,
                               const float* A, const float* B, const int32_t* perm, const float* node_proj,
                               int proj_stride, uint8_t* rec, size_t rec_stride, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t smem = sizeof(float) * ((size_t)R * d + 2 * (size_t)R * L + 4 * (size_t)R +
                                       (size_t)R * (L + 1) * m) +
                      sizeof(int32_t) * ((size_t)R + (size_t)R * (L + 1)) + sizeof(float) * (size_t)(L + 1) * m;
  cudaError_t e = cudaFuncSetAttribute(build_codes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, build_codes_kernel, kBuildThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)num_sms() * per_sm;
  if (grid > n) grid = n;
  build_codes_kernel<<<(unsigned)grid, kBuildThreads, smem, st>>>(X, n, d, nbrs, R, L, m, A, B, perm, node_proj,
                                                                  proj_stride, rec, rec_stride, code_bits(m),
                                                                  codes_per_word(m), code_words(L, m));
  return cudaGetLastError();
}

cudaError_t launch_node_proj(const float* X, int64_t n, int d, int L, int m, const float* A, const float* B,
                             const int32_t* perm, float* out, int out_stride, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const long long total = n * (long long)out_stride;
  long long grid = (total + 255) / 256;
  const long long cap = (long long)num_sms() * 16;
  if (grid > cap) grid = cap;
  node_proj_kernel<<<(unsigned)grid, 256, 0, st>>>(X, n, d, L, m, A, B, perm, out, out_stride);
  return cudaGetLastError();
}

cudaError_t launch_row_norms(const float* X, int64_t n, int d, float* norms, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  long long grid = (n + 255) / 256;
  const long long cap = (long long)num_sms() * 16;
  if (grid > cap) grid = cap;
  row_norms_kernel<<<(unsigned)grid, 256, 0, st>>>(X, n, d, norms);
  return cudaGetLastError();
}


namespace {
__global__ void wide_flags_kernel(const uint8_t* rec, size_t rec_stride, size_t ids_offset, long long n, int R,
                                  uint8_t* wide) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const int32_t* ids = reinterpret_cast<const int32_t*>(rec + (size_t)v * rec_stride + ids_offset);
    uint8_t any = 0;
    for (int s = 32; s < R; ++s) any |= (uint8_t)(ids[s] >= 0 && (long long)ids[s] < n);
    wide[v] = any;
  }
}
}  // namespace

cudaError_t launch_wide_flags(const uint8_t* rec, size_t rec_stride, size_t ids_offset, int64_t n, int R,
                              uint8_t* wide, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + 255) / 256, 4096);
  wide_flags_kernel<<<(unsigned)blocks, 256, 0, st>>>(rec, rec_stride, ids_offset, n, R, wide);
  return cudaGetLastError();
}

}  // namespace peos
