// Brute-force K-NN on the tensor cores (sm_103a tcgen05): the ground truth of the recall
// metric for large bases.
//
//   1. convert: base and queries to BF16 rows (zero-padded to a multiple of 64 elements),
//      and ||x||^2 of every base row in FP32;
//   2. candidates: per CTA (one per SM), a tile of 128 queries against one slice of the
//      base, the number of slices chosen by a cost model of waves, tiles and insertions.  A TMA warp brings
//      128 x 64 query and 256 x 64 base tiles (128-byte swizzled, K-major) into a ring of
//      2-4 shared-memory stages behind mbarriers; an MMA warp issues tcgen05.mma (BF16 in,
//      FP32 accumulate in tensor memory, M = 128, N = 256, K = 16 per instruction) into one
//      of two accumulators; four epilogue warps read the other accumulator with
//      tcgen05.ld, one query row per thread, screen 32 scores ||x||^2 - 2 q.x at a time
//      against the row's worst kept score (q's own norm does not change the order) and
//      insert the few that may enter the row's best `cand`, kept as a max-heap in shared
//      memory (the root is the worst kept key; an insertion replaces it and sifts down);
//   3. finalize: one warp per query takes the candidates of every slice, computes their
//      exact FP32 squared distances from the FP32 rows (sequential over the dimensions)
//      and keeps the k smallest by (dist, id).
// On integer-valued data below 256 (SIFT-shaped) the BF16 products and their FP32 sums
// are exact, so the candidates are exactly the best rows of each slice.  Otherwise the
// BF16 rounding only reorders near-ties, which the slack of `cand` over k absorbs; the
// final distances are always exact FP32.
//
// Every wait on an mbarrier is bounded: after kWaitLimitNs of the global timer (or
// kMaxPolls polls, whichever comes first) the CTA records an error and stops issuing work
// (the host reports PEOS_E_TIMEOUT).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "device.cuh"
#include "internal.h"

namespace peos {
namespace {

constexpr int kTcM = 128;      // queries per tile: accumulator rows = tensor-memory lanes
constexpr int kTcN = 256;      // base rows per tile: accumulator columns
constexpr int kTcK = 64;       // elements per stage: one 128-byte swizzle atom of BF16
constexpr int kMaxStages = 4;
constexpr int kEpiWarps = 4;                       // one per quarter of the tensor-memory lanes
constexpr int kEpiThreads = kEpiWarps * 32;        // = kTcM: one accumulator row per thread
constexpr int kTmaWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kTcThreads = (kEpiWarps + 2) * 32;
constexpr int kAccCols = 2 * kTcN;                 // two accumulators: all 512 tensor-memory columns
constexpr long long kWaitLimitNs = 2000000000ll;  // 2 s: no wait of a healthy launch comes near it
constexpr long long kMaxPolls = 1ll << 26;
constexpr int kMaxK = 96;          // k this path serves (candidates per slice: k + 16)
constexpr int kMaxCandTotal = 2048;  // candidates per query over all slices (finalize's shared memory)

constexpr int kABytes = kTcM * kTcK * 2;  // 16 KB
constexpr int kBBytes = kTcN * kTcK * 2;  // 32 KB

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// nanoseconds of the GPU's global timer
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of `bar` with the given parity; false when `limit_ns` nanoseconds of
// the global timer passed first.  The timer is read only once the first poll failed.
__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, uint32_t parity, long long limit_ns) {
  const uint32_t a = smem_u32(bar);
  uint64_t t0 = 0;
  for (long long i = 0; i < kMaxPolls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    const uint64_t t = global_ns();
    if (i == 0) t0 = t;
    else if ((long long)(t - t0) >= limit_ns) return false;
  }
  return false;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return mbar_wait_n(bar, parity, kWaitLimitNs);
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing arrives on;
// the wait gives up after `limit_ns` nanoseconds and the kernel records that it did.
__global__ void bounded_wait_probe_kernel(long long limit_ns, int* gave_up) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *gave_up = mbar_wait_n(&bar, 0, limit_ns) ? 0 : 1;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;            // start address
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused with swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                  // descriptor version
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, A and B K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// float -> unsigned with the same order (for keys that may be negative)
__device__ __forceinline__ uint32_t ordered(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// the score of a candidate key (inverse of ordered on the high word); +inf for an empty
// slot, so that every finite score may enter a list that is not full
__device__ __forceinline__ float key_score(uint64_t key) {
  if (key == kNoKey) return INFINITY;
  const uint32_t o = (uint32_t)(key >> 32);
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__global__ void convert_bf16_kernel(const float* __restrict__ X, long long n, int d, int pitch,
                                    __nv_bfloat16* __restrict__ out, float* __restrict__ norm2) {
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = w0; r < n; r += nw) {
    float s = 0.0f;
    for (int k = lane; k < pitch; k += 32) {
      const float v = k < d ? X[(size_t)r * d + k] : 0.0f;
      out[(size_t)r * pitch + k] = __float2bfloat16_rn(v);
      s += v * v;
    }
    if (norm2) {
      s = warp_sum(s);
      if (lane == 0) norm2[r] = s;
    }
  }
}

struct TcArgs {
  const float* xnorm;
  long long n, nq;
  int kchunks;       // pitch / 64
  int cand;          // candidates kept per query per slice
  long long slice;   // base rows per slice
  int nslice;
  int stages;        // shared-memory ring depth (2..kMaxStages)
  uint64_t* out;     // [nq][nslice][cand] (ordered(approx) << 32 | id)
  int* err;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void epilogue_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiWarps * 32) : "memory"); }

// Warp-specialised: warps 0-3 read the accumulator (each its quarter of the tensor-memory
// lanes, one query row per thread) and keep the candidates; warp 4 issues the TMA loads
// into a ring of `stages` shared-memory stages; warp 5 issues the MMAs into one of two
// accumulators (512 tensor-memory columns), so the MMAs of base tile t + 1 run while the
// epilogue reads tile t.
__global__ void __launch_bounds__(kTcThreads, 1) knn_tc_kernel(const __grid_constant__ CUtensorMap tq,
                                                                const __grid_constant__ CUtensorMap tx, TcArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  unsigned char* sm = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  const int S = a.stages;
  unsigned char* sA = sm;                                  // S x 16 KB
  unsigned char* sB = sA + S * kABytes;                    // S x 32 KB
  uint64_t* keys = reinterpret_cast<uint64_t*>(sB + S * kBBytes);  // [cand][128]
  uint64_t* bars = keys + (size_t)a.cand * kEpiThreads;    // full[S], empty[S], acc_full[2], acc_empty[2]
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* accf = bars + 2 * S;
  uint64_t* acce = accf + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  __shared__ volatile int s_fail;
  __shared__ volatile int s_efail[2];  // the epilogue's own failure flag, by tile parity
  __shared__ __align__(16) float s_xn[2][kTcN];  // ||x||^2 of the tile's base rows, double-buffered (read as float4)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long q0 = (long long)blockIdx.x * kTcM;
  const int sl = blockIdx.y;
  const long long r_begin = (long long)sl * a.slice;
  const long long r_end = min(a.n, r_begin + a.slice);
  const int ntiles = r_end > r_begin ? (int)((r_end - r_begin + kTcN - 1) / kTcN) : 0;

  if (tid == 0) {
    s_fail = 0;
    s_efail[0] = s_efail[1] = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf + b, 1);
      mbar_init(acce + b, kEpiThreads);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kAccCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < kEpiThreads)
    for (int i = 0; i < a.cand; ++i) keys[(size_t)i * kEpiThreads + tid] = kNoKey;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == kTmaWarp) {
    if (lane == 0) {
      uint32_t it = 0;
      for (int t = 0; t < ntiles && !s_fail; ++t) {
        const int r0 = (int)(r_begin + (long long)t * kTcN);
        for (int kc = 0; kc < a.kchunks; ++kc, ++it) {
          const int s = it % S;
          const uint32_t use = it / S;
          if (use > 0 && !mbar_wait(empty + s, (use - 1) & 1)) {
            s_fail = 1;
            break;
          }
          mbar_expect_tx(full + s, kABytes + kBBytes);
          tma_load_2d(sA + s * kABytes, &tq, full + s, kc * kTcK, (int)q0);
          tma_load_2d(sB + s * kBBytes, &tx, full + s, kc * kTcK, r0);
        }
      }
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kTcM, kTcN);
      uint32_t it = 0;
      for (int t = 0; t < ntiles && !s_fail; ++t) {
        const int b = t & 1;
        const uint32_t ub = (uint32_t)t >> 1;
        if (ub > 0 && !mbar_wait(acce + b, (ub - 1) & 1)) {  // the epilogue is done with this accumulator
          s_fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dacc = tmem + (uint32_t)(b * kTcN);
        bool ok = true;
        for (int kc = 0; kc < a.kchunks; ++kc, ++it) {
          const int s = it % S;
          const uint32_t use = it / S;
          if (!mbar_wait(full + s, use & 1)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int k16 = 0; k16 < kTcK / 16; ++k16) {
            const uint64_t da = smem_desc_sw128(sA + s * kABytes + k16 * 32);
            const uint64_t db = smem_desc_sw128(sB + s * kBBytes + k16 * 32);
            const uint32_t acc = (kc > 0 || k16 > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dacc),
                "l"(da), "l"(db), "r"(idesc), "r"(acc));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(empty + s))
                       : "memory");
        }
        if (!ok) {
          s_fail = 1;
          break;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(accf + b))
                     : "memory");
      }
    }
  } else {
    // epilogue: thread tid owns accumulator row tid (query q0 + tid); a score is compared
    // with the list's worst as a float first and becomes a key only when it may enter
    uint64_t* mine = keys + tid;
    for (int t = 0; t < ntiles; ++t) {
      const int b = t & 1;
      const long long r0 = r_begin + (long long)t * kTcN;
      for (int j = tid; j < kTcN; j += kEpiThreads) s_xn[b][j] = (r0 + j < r_end) ? __ldg(a.xnorm + r0 + j) : INFINITY;
      // a failed wait is flagged in this tile's slot before the barrier and read after it,
      // so all four warps leave together (a thread one tile ahead writes the other slot)
      if (!mbar_wait(accf + b, ((uint32_t)t >> 1) & 1)) {
        s_efail[b] = 1;
        s_fail = 1;
      }
      epilogue_sync();
      if (s_efail[b]) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint64_t worst = mine[0];  // the root of the row's max-heap of kept keys
      float worst_f = key_score(worst);
      for (int c0 = 0; c0 < kTcN; c0 += 32) {
        uint32_t v[32];
        __syncwarp();  // tcgen05.ld is warp-collective
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * kTcN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
            "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
            "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // screen 32 scores against the list's worst score: a bit per column that may enter.
        // Columns arrive in increasing order, so a score equal to the worst one has a larger
        // key than every kept key with that score and never enters: the test is strict.
        float sc[32];
        uint32_t mask = 0;
        const float4* xn4 = reinterpret_cast<const float4*>(&s_xn[b][c0]);
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
          const float4 xn = xn4[j4];
          sc[4 * j4 + 0] = __fmaf_rn(-2.0f, __uint_as_float(v[4 * j4 + 0]), xn.x);  // +inf past the slice
          sc[4 * j4 + 1] = __fmaf_rn(-2.0f, __uint_as_float(v[4 * j4 + 1]), xn.y);
          sc[4 * j4 + 2] = __fmaf_rn(-2.0f, __uint_as_float(v[4 * j4 + 2]), xn.z);
          sc[4 * j4 + 3] = __fmaf_rn(-2.0f, __uint_as_float(v[4 * j4 + 3]), xn.w);
#pragma unroll
          for (int u = 0; u < 4; ++u) mask |= (sc[4 * j4 + u] < worst_f ? 1u : 0u) << (4 * j4 + u);
        }
        // one set bit per lane per iteration, so lanes insert side by side (a single copy
        // of the insertion code; the score is picked out of the registers by selects)
        while (mask) {
          const int j = __ffs(mask) - 1;
          mask &= mask - 1;
          float sj = sc[0];
#pragma unroll
          for (int u = 1; u < 32; ++u) sj = (j == u) ? sc[u] : sj;
          const long long col = r0 + c0 + j;
          const uint64_t key = ((uint64_t)ordered(sj) << 32) | (uint32_t)col;
          if (col < r_end && key < worst) {
            // replace the heap's root (the worst kept key) and sift down
            int i = 0;
            for (;;) {
              const int l = 2 * i + 1;
              if (l >= a.cand) break;
              const int r = l + 1;
              const uint64_t hl = mine[(size_t)l * kEpiThreads];
              const uint64_t hr = r < a.cand ? mine[(size_t)r * kEpiThreads] : 0ull;
              const int c = (r < a.cand && hr > hl) ? r : l;
              const uint64_t hc = c == r ? hr : hl;
              if (hc <= key) break;
              mine[(size_t)i * kEpiThreads] = hc;
              i = c;
            }
            mine[(size_t)i * kEpiThreads] = key;
            worst = mine[0];
            worst_f = key_score(worst);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(acce + b);  // this thread is done with the accumulator
    }
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) atomicExch(a.err, 1);
  } else if (tid < kEpiThreads && q0 + tid < a.nq) {
    uint64_t* o = a.out + ((size_t)(q0 + tid) * a.nslice + sl) * a.cand;
    for (int i = 0; i < a.cand; ++i) o[i] = keys[(size_t)i * kEpiThreads + tid];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAccCols));
}

// Exact FP32 distances of every query's candidates (one warp per query, one candidate per
// lane at a time, a sequential sum over the dimensions), then the k smallest by (dist, id).
constexpr int kFinWarps = 4;
__global__ void __launch_bounds__(kFinWarps * 32) knn_tc_finalize(const float* __restrict__ X, const float* __restrict__ Q,
                                                                  long long nq, int d, const uint64_t* __restrict__ cand,
                                                                  int ncand, int P, int k, int32_t* __restrict__ ids_out,
                                                                  float* __restrict__ dists_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t* s_key = reinterpret_cast<uint64_t*>(smem_raw) + (size_t)warp * P;
  for (long long q = (long long)blockIdx.x * kFinWarps + warp; q < nq; q += (long long)gridDim.x * kFinWarps) {
    const float* qv = Q + (size_t)q * d;
    for (int i = lane; i < P; i += 32) {
      uint64_t key = kNoKey;
      if (i < ncand) {
        const uint64_t c = cand[(size_t)q * ncand + i];
        if (c != kNoKey) {
          const uint32_t id = (uint32_t)(c & 0xffffffffu);
          const float* xv = X + (size_t)id * d;
          float acc = 0.0f;
          for (int t = 0; t < d; ++t) {
            const float df = __ldg(qv + t) - __ldg(xv + t);
            acc = acc + df * df;
          }
          key = pack_key(acc, (int32_t)id);
        }
      }
      s_key[i] = key;
    }
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = lane; i < (P >> 1); i += 32) {
          const int lo = 2 * i - (i & (stride - 1));
          const int hi = lo + stride;
          const uint64_t x = s_key[lo], y = s_key[hi];
          if ((x > y) == ((lo & size) == 0)) {
            s_key[lo] = y;
            s_key[hi] = x;
          }
        }
        __syncwarp();
      }
    }
    for (int j = lane; j < k; j += 32) {
      const uint64_t key = s_key[j];
      ids_out[(size_t)q * k + j] = key == kNoKey ? -1 : key_id(key);
      dists_out[(size_t)q * k + j] = key == kNoKey ? INFINITY : key_dist(key);
    }
    __syncwarp();
  }
}

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiled encode_fn() {
  static std::mutex mu;
  static EncodeTiled fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

// 2-D tensor map over a BF16 matrix of `rows` rows of `pitch` elements; box = box_k x box_rows,
// 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, long long rows, int pitch, int box_rows) {
  EncodeTiled enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
  cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int knn_tc_pitch(int d) { return (d + kTcK - 1) / kTcK * kTcK; }

int knn_tc_cand(int k) { return k + 16; }

int knn_tc_slices(long long n, long long nq, int k, int sms) {
  // One CTA per SM; a CTA pays for its base tiles and for the insertions into its rows'
  // candidate heaps, about cand (1 + ln(rows / cand)) per row and slice (a random stream),
  // worth ~64 tiles of MMA and screening per unit of that log term (measured on GB300 at
  // d = 128 and 960).  Pick the slice count s minimising waves(s) x per-CTA cost, among
  // slices of >= 4 tiles and at most kMaxCandTotal candidates per query.
  const long long qt = (nq + kTcM - 1) / kTcM;
  const int cand = knn_tc_cand(k);
  long long max_s = (n + 4LL * kTcN - 1) / (4LL * kTcN);
  const long long max_c = kMaxCandTotal / cand;
  if (max_s > max_c) max_s = max_c;
  if (max_s < 1) max_s = 1;
  long long best = 1;
  double best_cost = -1.0;
  for (long long s = 1; s <= max_s; ++s) {
    const long long waves = (qt * s + sms - 1) / sms;
    const double rows = (double)((n + s - 1) / s);
    const double tiles = ceil(rows / kTcN);
    const double ins = rows > cand ? 1.0 + log(rows / cand) : 1.0;
    const double cost = (double)waves * (tiles + 64.0 * ins);
    if (best_cost < 0.0 || cost < best_cost) {
      best_cost = cost;
      best = s;
    }
  }
  return (int)best;
}

int knn_tc_max_k() { return kMaxK; }

size_t knn_tc_scratch_bytes(long long n, long long nq, int d, int k, int sms) {
  const size_t pitch = (size_t)knn_tc_pitch(d);
  const size_t ns = (size_t)knn_tc_slices(n, nq, k, sms);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return up((size_t)n * pitch * 2) + up((size_t)nq * pitch * 2) + up((size_t)n * 4) +
         up((size_t)nq * ns * knn_tc_cand(k) * 8) + 256;
}

cudaError_t launch_knn_tc(const float* X, long long n, int d, const float* Q, long long nq, int k, int32_t* ids_out,
                          float* dists_out, void* scratch, int* err_flag, cudaStream_t st) {
  (void)cudaGetLastError();  // start from a clean error state: the launch checks below read it
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int pitch = knn_tc_pitch(d);
  const int ns = knn_tc_slices(n, nq, k, sms);
  const int cand = knn_tc_cand(k);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  unsigned char* w = static_cast<unsigned char*>(scratch);
  __nv_bfloat16* xb = reinterpret_cast<__nv_bfloat16*>(w);
  w += up((size_t)n * pitch * 2);
  __nv_bfloat16* qb = reinterpret_cast<__nv_bfloat16*>(w);
  w += up((size_t)nq * pitch * 2);
  float* xnorm = reinterpret_cast<float*>(w);
  w += up((size_t)n * 4);
  uint64_t* cand_buf = reinterpret_cast<uint64_t*>(w);
  (void)err_flag;

  const int cg = sms * 8;
  convert_bf16_kernel<<<cg, 256, 0, st>>>(X, n, d, pitch, xb, xnorm);
  convert_bf16_kernel<<<cg, 256, 0, st>>>(Q, nq, d, pitch, qb, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  CUtensorMap mq, mx;
  if (!make_map(&mq, qb, nq, pitch, kTcM) || !make_map(&mx, xb, n, pitch, kTcN)) return cudaErrorNotSupported;
  TcArgs ta;
  ta.xnorm = xnorm;
  ta.n = n;
  ta.nq = nq;
  ta.kchunks = pitch / kTcK;
  ta.cand = cand;
  ta.slice = ((n + ns - 1) / ns + kTcN - 1) / kTcN * kTcN;
  ta.nslice = ns;
  ta.out = cand_buf;
  ta.err = err_flag;
  // as many ring stages as fit beside the candidate lists (at least 2, at most kMaxStages);
  // one CTA per SM either way (the two accumulators take all 512 tensor-memory columns)
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, knn_tc_kernel);
  if (e != cudaSuccess) return e;
  maxsm -= (int)fa.sharedSizeBytes;  // the kernel's static shared memory comes off the top
  const size_t fixed = 1024 + (size_t)cand * kEpiThreads * 8 + (2 * kMaxStages + 4) * 8 + 16;
  int stages = kMaxStages;
  while (stages > 2 && fixed + (size_t)stages * (kABytes + kBBytes) > (size_t)maxsm) --stages;
  size_t smem = fixed + (size_t)stages * (kABytes + kBBytes);
  if (smem > (size_t)maxsm) return cudaErrorInvalidConfiguration;
  const size_t one_per_sm = ((size_t)maxsm + fa.sharedSizeBytes) / 2 + 1024;  // never two CTAs on one SM
  if (smem < one_per_sm) smem = one_per_sm;
  ta.stages = stages;
  e = cudaFuncSetAttribute(knn_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((nq + kTcM - 1) / kTcM), (unsigned)ns);
  knn_tc_kernel<<<grid, kTcThreads, smem, st>>>(mq, mx, ta);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  const int ncand = ns * cand;
  int P = 1;
  while (P < ncand) P <<= 1;
  const size_t fsm = (size_t)P * 8 * kFinWarps;
  e = cudaFuncSetAttribute(knn_tc_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
  if (e != cudaSuccess) return e;
  long long fg = (nq + kFinWarps - 1) / kFinWarps;
  if (fg > (long long)sms * 8) fg = (long long)sms * 8;
  knn_tc_finalize<<<(unsigned)fg, kFinWarps * 32, fsm, st>>>(X, Q, nq, d, cand_buf, ncand, P, k, ids_out,
                                                             dists_out);
  return cudaGetLastError();
}

cudaError_t launch_bounded_wait_probe(long long limit_ns, int* gave_up, cudaStream_t st) {
  bounded_wait_probe_kernel<<<1, 32, 0, st>>>(limit_ns, gave_up);
  return cudaGetLastError();
}

}  // namespace peos
