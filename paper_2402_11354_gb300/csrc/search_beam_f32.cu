// The search kernel with beam width 2 and 4 (nodes expanded per iteration) over a base
// stored in FP32; compiled in its own translation unit so that the variants build in parallel.
#include "search_kernel.cuh"

namespace peos {
namespace sk {
template cudaError_t launch_search_beam<kF32, 1>(const KArgs&, int, int, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_search_beam<kF32, kMaxCodeWords>(const KArgs&, int, int, int, int, int, size_t, cudaStream_t);
}  // namespace sk
}  // namespace peos
