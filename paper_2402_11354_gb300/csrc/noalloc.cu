// Allocation-free search: the same kernels as peos_search, with their scratch in a
// fixed array that lives in the library's device image instead of memory taken
// from the device's pool.
//
// Some callers cannot call cudaMalloc or any allocating routine while they serve
// requests: engines that reserve all device memory up front and hand out only
// their own buffers, and latency-critical loops that must not take the
// allocator's locks or its implicit synchronisation.  They pass inputs and
// outputs as usual and the library uses the array below for everything else.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace peos {
namespace {

// Scratch of the allocation-free entry point: bytes [0, 256) hold the search's work
// counter, the rest any per-query scratch of the search.  The search needs none at
// present (each warp builds its query's projection table in shared memory), so no batch
// is rejected; the size check below stays for layouts that need per-query scratch.
// Every device that loads the library reserves this array until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)64 << 10;
constexpr size_t kNoAllocTableOffset = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the array on the current device: looked up on the first call
// on each device (with that device current) and cached.  The symbol's host-side
// name is not a device address and is never handed to a kernel.
peos_status scratch_on_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(PEOS_E_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PEOS_OK;
}

}  // namespace
}  // namespace peos

using namespace peos;

extern "C" {

peos_status peos_search_noalloc(const peos_graph* graph, peos_codes_t codes, const peos_matrix* base,
                                const peos_matrix* queries, const peos_search_params* params, int32_t* ids_out,
                                float* dists_out, int32_t* counters, void* stream) {
  NvtxRange nvtx_range("peos.search");
  peos_status st = check_matrix_public(queries, "queries");
  if (st) return st;
  SearchLaunch a;
  st = prepare_search(graph, codes, base, queries->n, queries->d, params, &a);
  if (st) return st;
  if (queries->n > 0 && (!ids_out || !dists_out)) return set_error(PEOS_E_INVAL, "NULL output");
  const size_t tables = search_scratch_bytes(queries->n, a.L, a.m, a.routing);
  if (tables > kNoAllocScratchBytes - kNoAllocTableOffset) {
    const size_t per_query = search_scratch_bytes(1, a.L, a.m, a.routing);
    return set_error(PEOS_E_INVAL, "query batch too large for the allocation-free scratch: at most " +
                                       std::to_string((kNoAllocScratchBytes - kNoAllocTableOffset) /
                                                      (per_query ? per_query : 1)) +
                                       " queries per call with these L and m");
  }
  unsigned char* scratch = nullptr;
  st = scratch_on_current_device(&scratch);
  if (st) return st;
  if (queries->n == 0) return PEOS_OK;
  a.Q = static_cast<const float*>(queries->data);
  a.ids_out = ids_out;
  a.dists_out = dists_out;
  a.counters = counters;
  a.work = reinterpret_cast<int*>(scratch);  // cleared by the launcher before the search kernel
  cudaError_t e = launch_search(a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "search launch");
  return PEOS_OK;
}

}  // extern "C"
