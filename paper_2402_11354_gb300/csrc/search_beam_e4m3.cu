// The search kernel with beam width 2 and 4 (nodes expanded per iteration) over a base
// stored in FP8 E4M3; compiled in its own translation unit so that the variants build in parallel.
#include "search_kernel.cuh"

namespace peos {
namespace sk {
template cudaError_t launch_search_beam<kE4M3, 1>(const KArgs&, int, int, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_search_beam<kE4M3, kMaxCodeWords>(const KArgs&, int, int, int, int, int, size_t, cudaStream_t);
}  // namespace sk
}  // namespace peos
