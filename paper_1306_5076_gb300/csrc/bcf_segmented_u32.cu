// bcf_segmented_u32.cu -- the persistent segmented sort instantiated for uint32_t keys.
#include "bcf_segmented.cuh"

namespace bcf {

template cudaError_t launch_segmented_typed<uint32_t>(bool, int, const SegArgs&, cudaStream_t);

}  // namespace bcf
