// The search kernel over a base stored in FP8 E4M3 (one FP32 scale per row); compiled in its own
// translation unit so that the element types build in parallel.
#include "search_kernel.cuh"

namespace peos {
namespace sk {
template cudaError_t launch_search_typed<kE4M3, 1>(const KArgs&, int, int, int, int, size_t, cudaStream_t);
}  // namespace sk
}  // namespace peos
