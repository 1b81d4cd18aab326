// The search kernel for codes of more than one 64-bit word per edge (L + 1 codes that do
// not fit one word, e.g. L = 24) over a base stored in FP32; compiled in its own
// translation unit so that the variants build in parallel.
#include "search_kernel.cuh"

namespace peos {
namespace sk {
template cudaError_t launch_search_typed<kF32, kMaxCodeWords>(const KArgs&, int, int, int, int, size_t, cudaStream_t);
}  // namespace sk
}  // namespace peos
