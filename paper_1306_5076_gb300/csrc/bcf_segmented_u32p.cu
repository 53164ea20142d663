// bcf_segmented_u32p.cu -- the persistent segmented sort instantiated for uint32_t keys
// with uint32_t payloads.
#include "bcf_segmented.cuh"

namespace bcf {

template cudaError_t launch_segmented_kp<uint32_t, true>(int, const SegArgs&, cudaStream_t);

}  // namespace bcf
