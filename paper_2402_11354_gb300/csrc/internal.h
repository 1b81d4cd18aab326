// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/peos.h"
#include "layout.h"

struct peos_codes_s {
  int device;
  int64_t n;
  int32_t R, L, m, d;
  int32_t entry;
  uint64_t seed;
  size_t rec_stride;   // bytes per node record
  uint8_t* records;    // n * rec_stride
  float* node_proj;    // n * table_stride(L, m)
  float* A;            // L * m * (d/L)
  float* B;            // m * d
  float* Wt;           // the same vectors k-major: B^T as [d][m], then a^i as [(i d/L + k)][m]
  int32_t* perm;       // dimension permutation (d entries) the codes and tables were built in, or null
  float* norms;        // ||v||^2 of every base row (sequential FP32 sums; frame Q), PEOs codes
  int kind;            // 0 = PEOs codes, 1 = SimHash bits (then L = 1, m = K, B = the K x d vectors,
                       // node_proj = n x K node table, A = Wt = null)
  int scalar_bits = 32;  // PEOs codes: width of the stored edge scalars (32, 16 or 8; layout.h)
  uint8_t* wide = nullptr;  // R > 32: per node, 1 if it has an edge in slots 32..R-1 (else null)
};

namespace peos {
// NVTX range over one library call ("peos.<call>"; no '/', which profilers read as
// nesting), so that a profiler can select the kernels one call launches by the range's
// name.  Without an attached tool the push and pop are a few instructions.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace peos

namespace peos {
constexpr int kCodesPeos = 0, kCodesSimHash = 1;
// floats per row of a handle's node table
inline int node_table_stride(const peos_codes_s* c) {
  return c->kind == kCodesSimHash ? c->m : table_stride(c->L, c->m);
}
}  // namespace peos

namespace peos {

// error plumbing (api.cu)
peos_status set_error(peos_status st, const std::string& msg);
peos_status cuda_error(cudaError_t e, const char* what);

// host random vectors (rng.cpp)
void projections_host(uint64_t seed, int d, int L, int m, float* A, float* B);

// launchers (build.cu)
cudaError_t launch_build_codes(const float* X, int64_t n, int d, const int32_t* nbrs, int R, int L, int m,
                               const float* A, const float* B, const int32_t* perm, const float* node_proj,
                               int proj_stride, uint8_t* rec, size_t rec_stride, cudaStream_t st);
cudaError_t launch_node_proj(const float* X, int64_t n, int d, int L, int m, const float* A, const float* B,
                             const int32_t* perm, float* out, int out_stride, cudaStream_t st);
cudaError_t launch_row_norms(const float* X, int64_t n, int d, float* norms, cudaStream_t st);
// the compact index: FP32 records (src) rewritten with 8- or 16-bit scalars (dst)
cudaError_t launch_compact_records(const uint8_t* src, size_t src_stride, int64_t n, int R, int words,
                                   const float* node_proj, int proj_stride, int L, int m, int sbits, uint8_t* dst,
                                   size_t dst_stride, cudaStream_t st);

// R > 32: per node, whether any of the record's ids in slots 32..R-1 is an edge (build.cu)
cudaError_t launch_wide_flags(const uint8_t* rec, size_t rec_stride, size_t ids_offset, int64_t n, int R,
                              uint8_t* wide, cudaStream_t st);
// attach those flags to a finished handle (api.cu); on failure the handle is unchanged
peos_status attach_wide_flags(peos_codes_s* c, cudaStream_t st);

// SimHash (simhash.cu): per-edge sign bits and ||e||, node table; thresholds on the host
cudaError_t launch_simhash_build(const float* X, int64_t n, int d, const int32_t* nbrs, int R, int K, const float* S,
                                 uint8_t* rec, size_t rec_stride, float* tv, cudaStream_t st);
void simhash_acrit(int K, double eps, float* acrit);

// dimension permutation (perm.cu): per-CTA partial sums of squared edge components, then
// the ordering and the greedy rounds in one CTA
size_t dim_perm_scratch_bytes(int d);
cudaError_t launch_dim_permutation(const float* X, int64_t n, int d, const int32_t* nbrs, int R, int L,
                                   void* scratch, int32_t* perm, cudaStream_t st);

// search (search.cu)
struct SearchLaunch {
  const void* X;          // stored base rows (dtype)
  const float* scales;    // per-row scales (FP8 E4M3), else null
  int dtype;              // peos_dtype of X
  const float* Xr;        // FP32 base for the exact re-rank of the final lists, or null
  int32_t* rr_ids;        // re-rank scratch: nq * ef ids and distances (when Xr)
  float* rr_dists;
  int64_t n;
  int d;
  const int32_t* nbrs;
  int R;
  int entry;
  const uint8_t* rec;
  size_t rec_stride;
  int tv_stride;  // floats per projection table row
  const float* A;
  const float* B;
  const float* Wt;  // k-major copy of the vectors (peos_codes_s::Wt)
  const int32_t* perm;  // dimension permutation of the codes (peos_codes_s::perm), or null
  int L, m;
  const float* Q;
  int64_t nq;
  int k, ef;
  int32_t* ids_out;
  float* dists_out;
  int32_t* counters;
  float z_eps, c_eta;
  int test_mode;
  int routing;
  int hash_bits;
  int hash_min_bits = 0;  // > 0: automatic table size, which the launcher may lower to this
  int max_exp;
  int warps_per_cta;
  int* work;       // device int, zeroed by the launcher on `st`
  int gather;      // rows per gather batch: 0 (routing default), 4 or 8
  int beam = 1;    // beam width W: nodes expanded per iteration (1, 2 or 4)
  const int32_t* k_q;   // uneven batches: per-query k (k = the maximum), or null
  const int32_t* ef_q;  // uneven batches: per-query efs (ef = the maximum), or null
  int32_t* order;       // scratch, nq ints: the batch order (used with ef_q)
  const int32_t* entries;  // per-query entry nodes, or null (entry)
  int frame;               // PEOs: 0 = frame T, 1 = frame Q (kernel variant ROUTING = 3)
  int scalar_bits;         // PEOs: width of the records' edge scalars (32; 16 / 8: variants 6 / 7)
  const float* norms;      // frame Q: squared norms of the base rows
  const uint8_t* wide;     // R > 32: per node, 1 if it has an edge in slots 32..R-1 (codes), or null
  // SimHash routing (routing = 2): K bits, node table n x K (B holds the K x d vectors),
  // and pass iff A <= acrit[#Col]
  int sh_K;
  const float* sh_tv;
  float sh_acrit[kMaxSimHashBits + 1];
};
cudaError_t launch_search(const SearchLaunch& a, cudaStream_t st);
#ifdef PEOS_CHECKED
unsigned long long* check_counters();  // self-checked builds: the current device's violation counters
#endif

// hierarchical entry (hier.cu): upper layers top first, device arrays
constexpr int kMaxHierLevels = 8;
struct HierLaunch {
  int levels;
  int top_entry;
  int64_t n[kMaxHierLevels];
  int R[kMaxHierLevels];
  const int32_t* ids[kMaxHierLevels];
  const int32_t* nbrs[kMaxHierLevels];
  const int32_t* down[kMaxHierLevels];
};
cudaError_t launch_hier_entry(const HierLaunch& h, const void* X, const float* scales, int dtype, int64_t nbase,
                              int d, const float* Q, int64_t nq, int* work, int32_t* entries, cudaStream_t st);
size_t search_smem_per_warp(int d, int ef, int hash_bits, int L, int m, int routing, int R, bool permuted, int beam);
size_t search_scratch_bytes(int64_t nq, int L, int m, int routing);
size_t search_rerank_smem(int d, int ef);

// reduced-precision storage (quant.cu)
cudaError_t launch_quantize(const float* X, int64_t n, int d, int dtype, void* out, float* scales, cudaStream_t st);

cudaError_t launch_edge_stats(const peos_codes_s* c, const float* q, int v, float dv, float delta2, float z_eps,
                              float c_eta, float* A_out, float* H_out, float* T_out, int32_t* pass_out,
                              int32_t* kind_out, cudaStream_t st);

// brute force (knn.cu)
size_t knn_scratch_bytes(int64_t n, int64_t nq, int k);
cudaError_t launch_knn(const float* X, int64_t n, int d, const float* Q, int64_t nq, int k, int32_t* ids_out,
                       float* dists_out, void* scratch, cudaStream_t st);

// stage tracing (api.cu): while tracing is on, each search records events around its
// stages (query tables, search kernel, re-rank) on its stream
struct TraceCall {
  cudaEvent_t ev[PEOS_NSTAGES + 1];
  int device;
};
bool trace_begin(TraceCall* tc);
void trace_end(const TraceCall& tc);

// brute force on the tensor cores (knn_tc.cu)
int knn_tc_max_k();
cudaError_t launch_bounded_wait_probe(long long limit_ns, int* gave_up, cudaStream_t st);
size_t knn_tc_scratch_bytes(long long n, long long nq, int d, int k, int sms);
cudaError_t launch_knn_tc(const float* X, long long n, int d, const float* Q, long long nq, int k, int32_t* ids_out,
                          float* dists_out, void* scratch, int* err_flag, cudaStream_t st);

// validation and launch description shared by the search entry points (api.cu)
peos_status prepare_search(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base, int64_t nq, int d_q,
                           const peos_search_params* P, SearchLaunch* a);
peos_status check_matrix_public(const peos_matrix* M, const char* name);

// host math for the test constants (api.cu)
double norm_ppf(double p);
double eta_value(int m, int mode);

}  // namespace peos
