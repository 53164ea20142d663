// bcf_segmented_u64p.cu -- the persistent segmented sort instantiated for uint64_t keys
// with uint32_t payloads.
#include "bcf_segmented.cuh"

namespace bcf {

template cudaError_t launch_segmented_kp<uint64_t, true>(int, const SegArgs&, cudaStream_t);

}  // namespace bcf
