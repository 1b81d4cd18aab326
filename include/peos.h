/*
 * peos.h -- C ABI of the GB300 (sm_103a) PEOs routing library.
 *
 * PEOs = Partitioned Extreme Order Statistics, the probabilistic routing test of
 * "Probabilistic Routing for Graph-Based Approximate Nearest Neighbor Search"
 * (arXiv 2402.11354).  The library runs batched graph beam search (Algorithm 1)
 * in which every out-edge of an expanded node is first screened by the PEOs test
 * (Sec. 4.2, Algorithm 2); exact l2 distances are computed only for the
 * neighbours that pass.
 *
 * Conventions for every entry point:
 *  - all buffers are owned by the caller unless stated otherwise; pointers marked
 *    "device" must be CUDA device memory on the current device, "host" pointers
 *    ordinary host memory;
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream);
 *    work is enqueued asynchronously on it, and host-side argument errors are
 *    returned before anything is enqueued;
 *  - the return value is a peos_status; on failure peos_last_error() gives a
 *    thread-local message;
 *  - matrices are row-major with rows of d contiguous elements; distances are
 *    squared l2 in FP32 (angular search = l2 on unit-normalised vectors, Sec. 2);
 *  - no entry point frees or retains caller memory after it returns, except that
 *    work enqueued on `stream` reads the caller's buffers until it completes.
 */
#ifndef PEOS_H
#define PEOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PEOS_OK = 0,
  PEOS_E_INVAL = 1,       /* an argument is out of range or inconsistent */
  PEOS_E_NOMEM = 2,       /* a device or host allocation failed */
  PEOS_E_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error string) */
  PEOS_E_OVERFLOW = 4,    /* per query: the expansion cap was reached before the search converged */
  PEOS_E_TIMEOUT = 5,     /* reserved for bounded device-side waits */
  PEOS_E_UNSUPPORTED = 6  /* valid but not implemented by this build (e.g. a dtype/d combination) */
} peos_status;

typedef enum { PEOS_F32 = 0, PEOS_BF16 = 1, PEOS_FP8E4M3 = 2 } peos_dtype;

/* Graph index G = (V, E) of Sec. 2: fixed out-degree R, nbrs[v*R + s] is the s-th
 * out-neighbour of v (-1 = empty slot).  nbrs is device memory, n*R int32. */
typedef struct {
  int64_t n;
  int32_t R;          /* 1..64 */
  int32_t entry;      /* entry node v_0 of Algorithm 1, 0 <= entry < n */
  const int32_t* nbrs;
} peos_graph;

/* n x d row-major matrix in device memory, d % 4 == 0, data 16-byte aligned.
 * dtype PEOS_F32: d floats per row, scales NULL.
 * dtype PEOS_BF16: d bfloat16 per row (value = the FP32 number with the same upper 16
 *   bits), scales NULL.
 * dtype PEOS_FP8E4M3: d bytes per row in the OCP FP8 E4M3 format (bias 7, no infinities,
 *   largest finite 448), and `scales` holds one FP32 scale per row (device, n floats):
 *   element k of row i stands for scales[i] * value(code[i][k]).
 * Only the base that a search reads may be BF16 or FP8E4M3 (the reduced-precision
 * storage of the precision form, produced by peos_quantize); queries, the base given to
 * peos_build_codes and peos_knn_bruteforce, and re-rank bases are PEOS_F32. */
typedef struct {
  const void* data;
  const float* scales;
  int64_t n;
  int32_t d;
  int32_t dtype;
} peos_matrix;

/* Library-owned index data built by peos_build_codes (device memory on the device
 * that was current at build time).  Released with peos_codes_free. */
typedef struct peos_codes_s* peos_codes_t;

typedef struct {
  int32_t k;              /* results per query, 1 <= k <= ef */
  int32_t ef;             /* size of the result list R of Algorithm 1 ("efs"), k <= ef <= 1024 */
  float eps;              /* error bound epsilon of Definition 3.1, 0 < eps <= 0.5 */
  int32_t routing;        /* 0 = plain (every unvisited neighbour is evaluated), 1 = PEOs test,
                             2 = SimHash test (codes from peos_build_simhash) */
  int32_t test_mode;      /* PEOs only: 0 = full test, 1 = only the A >= 1 / A <= 0 rules
                             (threshold T = -inf), 2 = every neighbour passes, 3 = full test with
                             the quantile lookup table of Sec. 4.3 (frame Q only): the variance
                             0 <= var <= L is taken at the upper edge of its bin of width 1/256
                             (256 L bins), a slightly smaller quantile */
  int32_t eta_mode;       /* 0 = eta = sqrt(2 ln m) (Lemma 4.2), 1 = finite-m mean of max_j |g_j| */
  int32_t max_expansions; /* per-query safety cap on expansions (<= 0: 1<<30) */
  int32_t visited_slots;  /* per-query visited-table slots, power of two 256..16384 (0 = auto: 16 efs,
                             clamped to 512..4096; where the shared memory of the tables, and not the
                             registers, limits the CTAs resident per SM, the largest of the halved
                             sizes, down to 512, that gives the most resident CTAs) */
  int32_t warps_per_cta;  /* queries resident per CTA, 1..8 (0 = auto) */
  int32_t gather_rows;    /* exact-distance rows gathered per batch: 4 or 8 (0 = the routing
                             method's default: 8 plain, 4 PEOs); results do not depend on it */
  const int32_t* entries; /* per-query entry nodes (nq int32, device; host for peos_search_host),
                             e.g. from peos_hier_entry, or NULL = graph.entry for every query.
                             A query whose entry is outside [0, n) returns an empty row and
                             PEOS_E_INVAL in its status counter.  Not accepted by the server. */
  int32_t frame;          /* PEOs (routing 1) only: 0 = frame T (translated by -v; the default),
                             1 = frame Q, the paper-literal form: the table of q' = q / ||q||
                             once per query and A_r = ((||u||^2/2 - r) - v.q) / (||q|| ||e||)
                             of Eq. A_r, r = ||p||^2/2 - p.q with p the list's efs-th entry; the
                             inner products come from the search's distances and the squared
                             norms (peos_codes_info.norms) by ||q - o||^2 = ||q||^2 + ||o||^2 -
                             2 q.o (Sec. 2); H is read straight from the table.  FP32 rows only. */
  int32_t beam;           /* beam width W, nodes expanded per iteration: 1 (Algorithm 1's pop-one
                             loop), 2 or 4 (0 = 1).  An iteration takes the W unexpanded entries of
                             R with the smallest (dist, id), freezes the list bound for the
                             iteration, tests their edges node after node (a neighbour that passed
                             earlier in the iteration counts as visited) and inserts all passes in
                             ascending (dist, id).  W > 1: plain routing, or PEOs in frame T with
                             FP32 scalars and no permutation (else PEOS_E_UNSUPPORTED). */
} peos_search_params;

/* Per-query counters written by peos_search when `counters` is non-NULL:
 * int32 [nq][PEOS_NCOUNTERS] in this order. */
enum {
  PEOS_C_EXPANSIONS = 0, /* nodes expanded (popped) */
  PEOS_C_EDGES,          /* valid out-edges of expanded nodes */
  PEOS_C_VISITED_SKIP,   /* out-edges whose head was found in the visited table */
  PEOS_C_A_REJECT,       /* PEOs: rejected because A >= 1 */
  PEOS_C_A_ACCEPT,       /* PEOs: accepted because A <= 0 */
  PEOS_C_H_TESTS,        /* PEOs: decided by H >= T */
  PEOS_C_H_PASS,         /* PEOs: ... and passed */
  PEOS_C_NDIST,          /* exact distances computed */
  PEOS_C_INSERTS,        /* insertions into R */
  PEOS_C_STATUS,         /* peos_status of the query (PEOS_OK or PEOS_E_OVERFLOW) */
  PEOS_C_FULL_EXPANSIONS, /* expansions made with |R| = ef (PEOs: the test read the edge weights/codes) */
  PEOS_NCOUNTERS
};

/* Build the PEOs index data (Sec. 4.2 steps (1)-(3), "pre-calculated during index
 * construction", Sec. 4.3):
 *   - the random vectors a^i_j ~ N(0, I_{d'}) (i = 1..L, j = 1..m, d' = d/L) and
 *     b_j ~ N(0, I_d) of step (2), drawn from `seed` by Philox4x64-10 + Box-Muller
 *     on the host (reproducible bit for bit, see peos_projections);
 *   - for every edge e = u - v: ||e||, w_reg = ||e_reg||/||e|| of step (1), the
 *     L+1 signed argmax codes e[0..L] of step (3), and the edge's node term
 *     sv = S(t(v)) of the statistic (below);
 *   - the projection table t(v) of every node (the vectors above applied to v).
 * The search's statistic needs the table of x = q - v, which is t(q) - t(v); its
 * code-selected weighted sum S(t) = w_reg sum_{c=1..L} sgn(e[c]) t[c][|e[c]|-1] +
 * sqrt(L) w_res sgn(e[0]) t[0][|e[0]|-1] is linear, so S(t(x)) = S(t(q)) - sv and the
 * search reads only t(q) (once per query) and sv (with the edge).
 * graph/base: device, as above; base must be PEOS_F32 with d % L == 0, d % 4 == 0.
 * L >= 1, 2 <= m <= 127.  Allocates device memory owned by the returned handle.
 * Enqueued on `stream`; the handle is usable by later work on the same stream. */
peos_status peos_build_codes(const peos_graph* graph, const peos_matrix* base, int32_t L, int32_t m,
                             uint64_t seed, void* stream, peos_codes_t* out);

/* Dimension permutation of Appendix D.1, computed on the device from the graph's edges:
 *   Avg(e_j) = (sum over the edges e = u - v, id >= 0, of e_j^2) / |E| in FP64 (0 if no edge);
 *   coordinates in ascending (Avg, j); then d/L rounds, round l giving coordinates of
 *   ranks (l-1)L .. lL-1, in that order, each to the subspace with the greatest running
 *   sum of Avg among those not yet given one in this round (equal sums: lower subspace);
 *   perm[i*(d/L) + t] = the original coordinate that becomes coordinate t of subspace i.
 * graph/base: device, base PEOS_F32 with d % L == 0 and d <= 2048.  perm: device array of
 * d int32 (caller-owned), written on `stream` (asynchronous; scratch is allocated and
 * released stream-ordered).  With integer-valued rows every sum is exact and the result
 * does not depend on the summation order. */
peos_status peos_dim_permutation(const peos_graph* graph, const peos_matrix* base, int32_t L, int32_t* perm,
                                 void* stream);

/* peos_build_codes in permuted coordinates (Appendix D.1): the edge vectors, their codes
 * and weights and the node tables are those of the rows with coordinate t read from
 * coordinate perm[t]; the search builds each query's table the same way.  The base and
 * the queries stay as they are (exact distances do not depend on the order of the
 * coordinates).  perm: device array of d int32, a permutation of 0..d-1 (checked:
 * PEOS_E_INVAL otherwise), copied into the handle; NULL = peos_build_codes. */
peos_status peos_build_codes_permuted(const peos_graph* graph, const peos_matrix* base, int32_t L, int32_t m,
                                      uint64_t seed, const int32_t* perm, void* stream, peos_codes_t* out);

/* The compact index: PEOs codes whose edge scalars (||e||, w_reg, sqrt(L) w_res) are
 * stored in scalar_bits = 16 or 8 bits instead of FP32 (the paper's 16-bit standard form
 * and 8-bit PEOs (Compact), Sec. 4.3 space analysis and Sec. 6.4; 32 = peos_build_codes).
 * Per node and scalar kind over the node's valid edges: s = max |x|, step =
 * s / (2^(bits-1) - 1), q = rint(x / step) clamped to the signed range (0 when step = 0),
 * and the test reads (float) q * step.  The node term stays FP32 and is recomputed from
 * the stored weights, so the statistic is that of the stored scalars.  The record shrinks
 * from 896 to 800 (16-bit) or 672 (8-bit) bytes per node at R = 32, L = 8, m = 16.
 * Searched with routing 1 in frame T over any stored type (frame Q: PEOS_E_UNSUPPORTED).
 * Synchronous on `stream`. */
peos_status peos_build_codes_compact(const peos_graph* graph, const peos_matrix* base, int32_t L, int32_t m,
                                     uint64_t seed, int32_t scalar_bits, void* stream, peos_codes_t* out);

/* Index data of the SimHash routing test (Sec. 3.1, Lemma 4.1; a baseline of the PEOs
 * test), with the residual remedy: for every edge e = u - v its K sign bits
 * [S_i . e >= 0] (sgn(0) = +1) and ||e||, for every node the table S_i . v, where S_i
 * (i < K) are the b_j of peos_projections(seed, d, 1, K).  Records use the layout of
 * peos_codes_info with scal = (||e||, 0, 0, 0) and the bits in K / 64 words (bit i in word
 * i / 64 at position i % 64); node_proj is the n x K table; L = 1, m = K.  All sums are
 * sequential FP32.  K = 64, 128 or 192.  Searched with routing = 2: in the frame
 * translated by -v, x = q - v has bits [S_i . q - S_i . v >= 0]; A as for PEOs (A >= 1
 * rejects, A <= 0 accepts); otherwise the edge passes iff A <= cos(pi (1 - (#Col + t) / K)),
 * #Col = K - popcount(bits(e) xor bits(x)), t = sqrt(K ln(1/eps) / 2) (Hoeffding's bound
 * on the binomial collision count; the cosine in FP64, rounded to FP32), 0 < eps < 1.
 * SimHash searches read FP32 rows. */
peos_status peos_build_simhash(const peos_graph* graph, const peos_matrix* base, int32_t K, uint64_t seed,
                               void* stream, peos_codes_t* out);

/* Release a handle from peos_build_codes (synchronises its device first). NULL is a no-op. */
peos_status peos_codes_free(peos_codes_t codes);

/* Read-only view of a handle's device arrays (for tests and tools).
 * records: n rows of `record_stride` bytes; row v holds, for s = 0..R-1:
 *   float4 scal[R] = (enorm, wreg, cres, sv) at byte 0 | int32 ids[R] at byte 16R |
 *   uint64 codes[W][R] at byte 20R rounded up to a multiple of 16 (then padding);
 *   with scalar_bits 16 or 8 (the compact index) the scalars are instead the node's
 *   float4 of steps (enorm, wreg, cres, 0) at byte 0, then per edge q = (q_enorm, q_wreg,
 *   q_cres, 0) (scalar = (float) q * step) and the FP32 node term sv: 16-bit as float
 *   sv[R] at byte 16 and short4 q[R] at byte 16 + 4R rounded up to a multiple of 8;
 *   8-bit as pairs {char4 q, float sv}[R] at byte 16; the ids right after and the codes
 *   at the next multiple of 16;
 *   enorm = ||e||, wreg = w_reg, cres = sqrt(L) w_res with w_res = sqrt(1 - w_reg^2),
 *   sv = the node term S(t(v)) summed in order c = 1..L then weighted as w_reg*h1 + cres*h2;
 *   codes: e[c] of edge s (c = 0 over the b_j with e_res, c = i over the a^i_j with e_i) in
 *   B = ceil(log2 m) + 1 bits as (|e[c]| - 1) | (e[c] < 0) << (B - 1); code c sits in word
 *   c / (64 / B) at bit (c % (64 / B)) * B; W = ceil((L + 1) / (64 / B)) <= 3.
 * node_proj: n rows of node_proj_stride floats (= (L+1)*m rounded up to a multiple of 4, zero
 *   padded); entry c*m + j of row v is b_j . v (c = 0) or a^c_j . v_c (c >= 1).
 * A: L x m x d' floats, B: m x d floats (device).
 * perm: the handle's dimension permutation (d int32, device) or NULL.
 * kind: 0 = PEOs codes (peos_build_codes), 1 = SimHash bits (peos_build_simhash).
 * norms: PEOs codes: ||v||^2 of every base row (n floats, sequential FP32 sums; frame Q).
 * scalar_bits: PEOs codes: width of the records' edge scalars (32, or 16 / 8 for the
 * compact index of peos_build_codes_compact); 32 for SimHash bits. */
typedef struct {
  int64_t n;
  int32_t R, L, m, d;
  int32_t entry;
  size_t record_stride;
  int32_t node_proj_stride;
  const uint8_t* records;
  const float* node_proj;
  const float* A;
  const float* B;
  const int32_t* perm;
  int32_t kind;
  const float* norms;
  int32_t scalar_bits;
} peos_codes_info;
peos_status peos_codes_get_info(peos_codes_t codes, peos_codes_info* info);

/* Copy a handle's arrays to host memory (synchronous on the handle's device):
 * records_host n*record_stride bytes (the record form of the handle's scalar width; see
 * peos_build_codes_compact), node_proj_host n*node_proj_stride floats, A_host
 * L*m*(d/L) floats, B_host m*d floats.  Any output may be NULL (skipped). */
peos_status peos_codes_export(peos_codes_t codes, void* records_host, float* node_proj_host, float* A_host,
                              float* B_host);

/* Batched graph search, Algorithm 1 with the readings below, plain or with the
 * PEOs test of Algorithm 2 (Sec. 4.2 steps (4)-(6)):
 *   - R is kept sorted by (dist, id); the unexpanded entry with the smallest
 *     (dist, id) is expanded next; the search ends when every entry of R is expanded;
 *   - delta and |R| = ef are frozen at the start of an expansion; the neighbours
 *     that pass are evaluated exactly, sorted by (dist, id) and inserted in order,
 *     each only if |R| < ef or dist < delta of the list as it stands;
 *   - a neighbour is visited only once its exact distance is computed (Sec. 3.1's
 *     residual remedy lets a rejected neighbour pass later from another node);
 *   - PEOs test in the frame translated by -v: with x = q - v, A = (||x||^2 +
 *     ||e||^2 - delta^2) / (2 ||x|| ||e||) (Eq. A_r after translation); A >= 1 rejects,
 *     A <= 0 accepts, otherwise pass iff H >= T with
 *     H = (S(t(q)) - sv) / ||x|| (step 5 on the table of x = q - v, see
 *     peos_build_codes) and
 *     T = A sqrt(L) eta + Phi^{-1}(eps) sqrt(w_reg^2 + L w_res^2 - L A^2/(L+1))
 *     (the eps-quantile of Eq. N_ex_min), decided without the square root as
 *     (A c - H <= 0) or ((A c - H)^2 <= Phi^{-1}(eps)^2 var) since Phi^{-1}(eps) <= 0;
 *   - each warp builds its query's projection table t(q) in shared memory (each entry
 *     stored with its negation, so a code indexes its signed term directly); the call
 *     takes a few hundred bytes of stream-ordered scratch (the work counter) from the
 *     device's default memory pool (cudaMallocAsync); the library sets that pool's
 *     release threshold to the maximum on first use so freed scratch stays mapped for
 *     the next call (peos_release_workspace trims it);
 *   - codes may be NULL for routing = 0.
 * base: PEOS_F32, PEOS_BF16 or PEOS_FP8E4M3 (distances are then taken to the widened,
 * scaled rows, accumulated in FP32); codes must have been built from the FP32 rows.
 * queries: device PEOS_F32, nq x d (same d as base; nq may be 0).
 * ids_out [nq][k] int32 and dists_out [nq][k] float: device; results in ascending
 * (dist, id); -1 / +inf pad when fewer than k nodes were reached.
 * counters: device int32 [nq][PEOS_NCOUNTERS] or NULL.
 * Returns PEOS_OK once the launch is enqueued; per-query overflow of the
 * expansion cap is reported in counters[.][PEOS_C_STATUS]. */
peos_status peos_search(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                        const peos_matrix* queries, const peos_search_params* params, int32_t* ids_out,
                        float* dists_out, int32_t* counters, void* stream);

/* peos_search followed by an exact FP32 re-rank of each query's final list R (the
 * precision form: the search ranks by distances to reduced-precision rows, the answer by
 * exact ones).  After the search, every entry of R (|R| <= ef) gets its squared l2
 * distance recomputed from `rerank` (device PEOS_F32, same n and d as base), R is sorted
 * again by (dist, id) and the first k are written to ids_out/dists_out.  rerank = NULL
 * gives exactly peos_search.  Scratch as peos_search plus nq * ef * 8 bytes for the lists.
 * Counters describe the search; the re-rank computes |R| further distances per query
 * that PEOS_C_NDIST does not include. */
peos_status peos_search_rerank(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                               const peos_matrix* rerank, const peos_matrix* queries,
                               const peos_search_params* params, int32_t* ids_out, float* dists_out,
                               int32_t* counters, void* stream);

/* Uneven batches in one launch, without allocation (CUDA-graph capturable).
 * Query i is searched with its own efs = ef_per_query[i] and returns its own
 * k_i = k_per_query[i] results (device int32 arrays of nq, or NULL = params->ef /
 * params->k for every query); params->ef and params->k are the maxima, which size the
 * per-query shared memory and the output rows: ids_out/dists_out are [nq][params->k],
 * slots >= k_i hold -1 / +inf.  A query with k_i or efs_i out of range (k_i < 1,
 * k_i > params->k, efs_i < k_i, efs_i > params->ef) gets an empty row and, when counters
 * are requested, PEOS_E_INVAL in its status counter.  Queries are taken in descending
 * efs order so that the persistent CTAs finish together.  rerank: as in
 * peos_search_rerank (NULL = none).
 * workspace: caller-owned device memory of at least peos_search_batch_workspace_size()
 * bytes (256-byte aligned); the call allocates nothing, so it can be captured into a
 * CUDA graph (make one call outside the capture first) and replayed.  Calls that share a
 * workspace must not overlap on the GPU. */
peos_status peos_search_batch_workspace_size(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                                             const peos_matrix* rerank, int64_t nq,
                                             const peos_search_params* params, size_t* bytes);
peos_status peos_search_batch(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                              const peos_matrix* rerank, const peos_matrix* queries,
                              const peos_search_params* params, const int32_t* k_per_query,
                              const int32_t* ef_per_query, int32_t* ids_out, float* dists_out, int32_t* counters,
                              void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------------
 * Serving: continuous batching with admission by device memory (the paper has no
 * counterpart; this is the deployment form of the search).
 *
 * A server keeps graph, codes and base resident (the caller's buffers, which must
 * outlive it).  Requests -- one query (host memory, copied at submission), its k and
 * its efs -- enter a host queue.  A scheduler thread takes batches of up to max_batch
 * requests from the queue head and runs each with peos_search_batch on one of
 * `streams` CUDA streams, so up to `streams` batches are on the GPU at once and requests
 * that arrive meanwhile are admitted as soon as a stream and device memory are free.
 * Each batch takes one contiguous range of a device arena of memory_budget bytes for its
 * queries, per-query k and efs, results and search workspace (query tables, re-rank
 * lists); a batch is admitted only if the arena has room (first fit; the batch is halved
 * until it fits, and waits when even one request does not).  The per-query on-chip state
 * (result list, visited table) is bounded by k_max / ef_max through the launch shape.
 * A request's result depends only on the request: it is the same alone and in any mix.
 * Times are steady-clock nanoseconds since the server was created. */
typedef struct peos_server_s* peos_server_t;
typedef struct {
  int32_t max_batch;           /* requests per launch, >= 1 */
  int32_t streams;             /* batches in flight at once, 1..16 */
  size_t memory_budget;        /* device bytes of the request arena */
  int32_t k_max, ef_max;       /* bounds of the requests' k and efs */
  peos_search_params params;   /* routing, eps, eta_mode, launch shape (k and ef are ignored) */
} peos_server_config;
typedef struct {
  uint64_t request_id;
  int32_t k;                   /* results in the row (the request's k) */
  int32_t status;              /* PEOS_OK, or the failure of the request's batch */
  int64_t arrival_ns, admit_ns, complete_ns;
} peos_server_result;
typedef struct {
  uint64_t submitted, completed, failed, pending;
  uint64_t batches, batched_queries, admission_waits;
  size_t arena_bytes, arena_used, arena_peak;
  int32_t batches_in_flight;
  int32_t last_error;
} peos_server_stats_t;

/* Create a server on the current device.  base/rerank/codes/graph as for
 * peos_search_batch (rerank may be NULL); d = base->d (the host query length). */
peos_status peos_server_create(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                               const peos_matrix* rerank, int32_t d, const peos_server_config* cfg,
                               peos_server_t* out);
/* Queue one request now (query: host, d floats; copied before returning). */
peos_status peos_server_submit(peos_server_t server, uint64_t request_id, const float* query, int32_t k, int32_t ef);
/* Start a load generator thread that submits request i at arrival_ns[i] nanoseconds
 * after this call (ascending offsets; all arrays host, copied before returning). */
peos_status peos_server_replay(peos_server_t server, int64_t n, const uint64_t* request_ids, const float* queries,
                               const int32_t* k, const int32_t* ef, const int64_t* arrival_ns);
/* Take up to max_results finished requests in completion order: results[i], and their
 * ids/dists rows of k_max entries in ids_out/dists_out (host); waits up to wait_us for
 * the first one when none is ready.  *n_out = the number returned. */
peos_status peos_server_poll(peos_server_t server, int32_t max_results, peos_server_result* results,
                             int32_t* ids_out, float* dists_out, int32_t* n_out, int32_t wait_us);
peos_status peos_server_stats(peos_server_t server, peos_server_stats_t* out);
/* Stop the generator and scheduler, wait for batches in flight, free the server. */
peos_status peos_server_destroy(peos_server_t server);

/* Reduced-precision copy of an FP32 matrix (device src, n x d): dtype PEOS_BF16 writes
 * n*d bfloat16 values rounded to nearest (ties to even) into data_out (scales_out may be
 * NULL; if given, it is filled with 1); PEOS_FP8E4M3 writes n*d E4M3 codes of
 * x * (448 / max|x_row|) rounded to nearest (ties to even, saturated to 448) and the
 * per-row scale max|x_row| / 448 (1 for an all-zero row) into scales_out (n floats).
 * All buffers device memory; enqueued on `stream`. */
peos_status peos_quantize(const peos_matrix* src, int32_t dtype, void* data_out, float* scales_out, void* stream);

/* Same search with the queries and results in HOST memory: copies the queries to
 * the device, searches, copies ids/dists (and counters when non-NULL) back, and
 * synchronises `stream` before returning.  The device staging area comes from the
 * stream-ordered pool (kept for reuse until peos_release_workspace). */
peos_status peos_search_host(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                             const float* queries_host, int64_t nq, const peos_search_params* params,
                             int32_t* ids_host, float* dists_host, int32_t* counters_host, void* stream);

/* peos_search_host without the final synchronisation: the copies in, the search and the
 * copies out are enqueued on `stream` and the call returns.  The host buffers must be
 * page-locked (cudaHostAlloc / pinned) for the copies to run asynchronously, and must not
 * be written (queries) or read (results) until `stream` has been synchronised.  Calls on
 * two streams overlap one batch's copies with another batch's search. */
peos_status peos_search_host_async(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                                   const float* queries_host, int64_t nq, const peos_search_params* params,
                                   int32_t* ids_host, float* dists_host, int32_t* counters_host, void* stream);

/* peos_search without any device allocation (the paper has no counterpart: this is a
 * deployment aid).  For callers that must not allocate while they serve requests,
 * e.g. engines that reserve all device memory up front and hand out only their own
 * buffers, or latency-critical loops that cannot take the allocator's locks and
 * implicit synchronisation.  Arguments, outputs and results are those of
 * peos_search; the search's scratch (its work counter) lives in a fixed 64 KiB array in
 * the library's device image, which every device that loads the library holds until the
 * process exits.
 *  - Limit: none at present -- the search needs no per-query device scratch (each warp
 *    builds its query's projection table in shared memory).  A batch whose per-query
 *    scratch would not fit the array is rejected with PEOS_E_INVAL before anything is
 *    enqueued.
 *  - The first call on a device looks up the array's device address (with that device
 *    current); make that first call before any stream capture.
 *  - Every call on a device shares the one array: calls whose work overlaps on the GPU
 *    (different streams without ordering between them) race and give wrong results.
 *    The work counter is cleared at the start of each call, so consecutive calls are
 *    independent.
 *  - Calls no cudaMalloc, cudaMallocAsync, cudaFree or other allocating routine. */
peos_status peos_search_noalloc(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                                const peos_matrix* queries, const peos_search_params* params, int32_t* ids_out,
                                float* dists_out, int32_t* counters, void* stream);

/* Free the library's cached per-device staging memory (synchronises the device). */
peos_status peos_release_workspace(void);

/* The PEOs statistics of every out-edge of one node for one query, by the same
 * device code the search uses (diagnostics and parity tests): query q (device,
 * d floats), expanded node v whose stored exact distance is dv = ||q - v||^2,
 * list bound delta2 (a full list).  Outputs (device, R each): A, H, T (0 where not
 * evaluated), pass (0/1) and kind (0 = A >= 1, 1 = A <= 0, 2 = H >= T decided,
 * 3 = degenerate edge or x = 0 accepted).  PEOs codes with FP32 scalars only
 * (PEOS_E_UNSUPPORTED for the compact index). */
peos_status peos_edge_stats(peos_codes_t codes, const float* query, int32_t v, float dv, float delta2,
                            float eps, int32_t eta_mode, float* A_out, float* H_out, float* T_out,
                            int32_t* pass_out, int32_t* kind_out, void* stream);

/* The random vectors of Sec. 4.2 step (2) for (seed, d, L, m), computed on the host
 * (no device work): A_host L x m x (d/L) floats, B_host m x d floats.  Philox4x64-10
 * keyed by (seed, tag); counter (column/4, row, matrix, 0); two Box-Muller pairs per
 * block in FP64, each rounded once to FP32. */
peos_status peos_projections(uint64_t seed, int32_t d, int32_t L, int32_t m, float* A_host, float* B_host);

/* Hierarchical entry (the paper's HNSW indexes, Sec. 6.1): upper layers over subsets of
 * the base, each a graph of its own nodes, searched top down by greedy search with a
 * list of one; the node reached in the lowest upper layer is the query's entry node for
 * the search on the base graph (peos_search_params.entries).
 * A layer (device arrays, caller-owned): n nodes; ids[i] = base row of local node i;
 * nbrs[i*R + s] = local ids (-1 empty), R <= 32; down[i] = the node's local id in the next
 * lower upper layer (NULL on the lowest).  layers: host array, top layer first, 1..8 of
 * them; every walk starts at local node top_entry of the top layer. */
typedef struct {
  int64_t n;
  int32_t R;
  const int32_t* ids;
  const int32_t* nbrs;
  const int32_t* down;
} peos_layer;
typedef struct {
  int32_t levels;
  const peos_layer* layers;
  int32_t top_entry;
} peos_hierarchy;

/* The entry node of every query (entries: nq int32, device).  At the current node c of a
 * layer, the neighbour with the smallest (exact squared l2 distance, base id) is taken if
 * it is strictly closer than c, else the walk moves down (through `down`) or ends.
 * Distances are to the rows of `base` (any stored type, as for peos_search) and reduce
 * across the warp as in the search.  Ids that leave their layer or the base end the walk
 * with entry -1 (the search then rejects that query).  Enqueued on `stream`. */
peos_status peos_hier_entry(const peos_hierarchy* hierarchy, const peos_matrix* base, const peos_matrix* queries,
                            int32_t* entries, void* stream);

/* Self-test of the failure detection of the library's waits: every spin-wait in the
 * device code (the tensor-core brute force's mbarrier waits) gives up after a bounded
 * time (2 s of the GPU's global timer), records the failure and returns (the host then
 * reports PEOS_E_TIMEOUT) instead of hanging.  This runs one such wait, limited to
 * `limit_us` microseconds (1..2,000,000), on an mbarrier that nothing arrives on,
 * synchronises `stream`, and sets *gave_up (host) to 1 when the wait gave up as it must.
 * Nothing faults or hangs; the context stays usable. */
peos_status peos_selftest_bounded_wait(int64_t limit_us, int32_t* gave_up, void* stream);

/* Exact K nearest neighbours by brute force (the ground truth of the recall metric):
 * for each query the k base rows with the smallest squared l2 distance, ascending
 * (dist, id).  Distances are exact FP32 sums of squared differences.
 * base/queries: device PEOS_F32; ids_out [nq][k], dists_out [nq][k] device;
 * 1 <= k <= 256.  Uses library-owned scratch of at most about 1 GiB (the queries run in
 * slices whose per-chunk candidate lists fit in it). */
peos_status peos_knn_bruteforce(const peos_matrix* base, const peos_matrix* queries, int32_t k,
                                int32_t* ids_out, float* dists_out, void* stream);

/* Device-time tracing of the search stages (diagnostics and the benchmark's roofline).
 * Stages: set-up (the descending-efs order of an uneven batch), the search kernel, the
 * FP32 re-rank.  While tracing is on, every search call records CUDA events on its
 * stream around its stages; peos_trace_read waits for the traced calls, adds up the device time of each
 * stage since the last read (ms[PEOS_NSTAGES], host) and the number of calls (host), and
 * starts a new tally.  Stages that a call does not run count 0 ms.  Tracing adds one
 * event record per stage to each call; it is off by default. */
enum { PEOS_STAGE_SETUP = 0, PEOS_STAGE_SEARCH, PEOS_STAGE_RERANK, PEOS_NSTAGES };
peos_status peos_trace_enable(int32_t on);
peos_status peos_trace_read(double* ms, int64_t* calls);

/* The same K-NN on the tensor cores (tcgen05, BF16 inputs, FP32 accumulation in tensor
 * memory) for large bases: every base row is scored by ||x||^2 - 2 q.x for every query,
 * each query keeps its k + 16 best rows per slice of the base, and those candidates get
 * their exact FP32 squared distances (sequential over the dimensions) and are ranked by
 * (dist, id).  On integer-valued data below 256 the BF16 scores are exact and the result
 * is the exact K-NN; otherwise BF16 rounding can only reorder near-ties among rows the
 * slack does not cover.  1 <= k <= 96.  Synchronous: returns after the results are
 * written (PEOS_E_TIMEOUT if a CTA's bounded wait for its tiles gave up). */
peos_status peos_knn_tensor(const peos_matrix* base, const peos_matrix* queries, int32_t k, int32_t* ids_out,
                            float* dists_out, void* stream);

/* ---- index files ------------------------------------------------------------------
 * A codes handle (PEOs codes of peos_build_codes / peos_build_codes_permuted, or SimHash
 * bits of peos_build_simhash) is written to a file and read back, so an index is built
 * once and searched from other processes.  The graph travels inside the edge records
 * (peos_codes_graph reads it back out); the base vectors are the caller's and are not
 * part of the file.  Layout (little-endian): the 8 bytes "PEOSIDX1",
 * a header with the handle's kind, n, R, L, m, d, entry, seed and strides, a table of
 * sections (id, CRC-32, bytes), the CRC-32 of header and table, then the sections
 * (records, node tables, A, B, Wt, the permutation, the row norms: those the handle has)
 * byte for byte as they sit in device memory.  CRC-32 is the zlib / IEEE 802.3 one. */

/* CRC-32 of `bytes` bytes at `data` (host) into *out (host). */
peos_status peos_crc32(const void* data, size_t bytes, uint32_t* out);

/* Write `codes` to `path` (created or truncated).  Synchronises the handle's device
 * first; the handle is unchanged.  PEOS_E_INVAL when the file cannot be written (a
 * partial file may be left behind). */
peos_status peos_codes_save(peos_codes_t codes, const char* path);

/* Read a file written by peos_codes_save into a new handle on the current device (free
 * it with peos_codes_free).  Every field is checked before use: the magic and version,
 * the header's CRC, a shape the builders accept, strides and section sizes that follow
 * from that shape, the set of sections the kind needs, each section's CRC and, for the
 * permutation, that it is one.  Any failure (a truncated, corrupted or foreign file)
 * returns PEOS_E_INVAL with *out = NULL and nothing allocated; PEOS_E_NOMEM when host or
 * device memory runs out.  Synchronous. */
peos_status peos_codes_load(const char* path, peos_codes_t* out);

/* The graph an index was built on, from the edge ids its records hold: nbrs (device,
 * n x R int32, row-major, -1 for empty slots) and *entry (host).  With a loaded index
 * file this gives the graph argument of peos_search.  Enqueued on `stream`. */
peos_status peos_codes_graph(peos_codes_t codes, int32_t* nbrs, int32_t* entry, void* stream);

/* ---- self-checked builds --------------------------------------------------------
 * The library built with -DPEOS_CHECKED checks, in the search kernel, every index it
 * computes before using it (a passing neighbour's id and its slot among the candidates,
 * the expanded node, every write position in the list) and, after every merge, that the
 * list is strictly ascending in (dist, id) and holds no id twice.  A violation is counted
 * by kind and the access is skipped (a bug shows up as a count, not as a fault).  Results
 * are identical to the normal build's.  peos_check_read synchronises the current device,
 * copies its PEOS_CHECK_KINDS counters to `counts` (host) and zeroes them; a normal build
 * returns PEOS_E_UNSUPPORTED (counts all 0).  Kinds: 0 candidate id or slot, 1 expanded
 * node, 2 list write position, 3 list order, 4 duplicate id in the list. */
#define PEOS_CHECK_KINDS 8
peos_status peos_check_read(uint64_t* counts);

/* Thread-local description of the last error returned on this thread. */
const char* peos_last_error(void);

/* Library version string. */
const char* peos_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PEOS_H */
