// The search kernel over a base stored in BF16 (unscaled rows); compiled in its own
// translation unit so that the element types build in parallel.
#include "search_kernel.cuh"

namespace peos {
namespace sk {
template cudaError_t launch_search_typed<kBF16, 1>(const KArgs&, int, int, int, int, size_t, cudaStream_t);
}  // namespace sk
}  // namespace peos
