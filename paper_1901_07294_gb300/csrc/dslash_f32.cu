// Hop kernel instantiations for one storage precision (compiled as its own
// translation unit so the precisions build in parallel).
#include "dslash_launch.cuh"

namespace wd {
template cudaError_t launch_hop<PREC_F32>(const HopArgs &, int, int, int, int, int, cudaStream_t);
} // namespace wd
