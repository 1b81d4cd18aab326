// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

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
};

namespace peos {

// error plumbing (api.cu)
peos_status set_error(peos_status st, const std::string& msg);
peos_status cuda_error(cudaError_t e, const char* what);

// host random vectors (rng.cpp)
void projections_host(uint64_t seed, int d, int L, int m, float* A, float* B);

// launchers (build.cu)
cudaError_t launch_build_codes(const float* X, int64_t n, int d, const int32_t* nbrs, int R, int L, int m,
                               const float* A, const float* B, const float* node_proj, int proj_stride,
                               uint8_t* rec, size_t rec_stride, cudaStream_t st);
cudaError_t launch_node_proj(const float* X, int64_t n, int d, int L, int m, const float* A, const float* B,
                             float* out, int out_stride, cudaStream_t st);

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
  int max_exp;
  int warps_per_cta;
  int* work;       // device int, zeroed by the launcher on `st`
  int gather;      // rows per gather batch: 0 (routing default), 4 or 8
  const int32_t* k_q;   // uneven batches: per-query k (k = the maximum), or null
  const int32_t* ef_q;  // uneven batches: per-query efs (ef = the maximum), or null
  int32_t* order;       // scratch, nq ints: the batch order (used with ef_q)
};
cudaError_t launch_search(const SearchLaunch& a, cudaStream_t st);
size_t search_smem_per_warp(int d, int ef, int hash_bits, int L, int m, int routing, int R);
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
