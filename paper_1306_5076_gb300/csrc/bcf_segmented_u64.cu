// bcf_segmented_u64.cu -- the persistent segmented sort instantiated for uint64_t keys.
#include "bcf_segmented.cuh"

namespace bcf {

template cudaError_t launch_segmented_typed<uint64_t>(bool, int, const SegArgs&, cudaStream_t);

}  // namespace bcf
