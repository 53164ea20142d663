// bcf_segmented_u64.cu -- the persistent segmented sort instantiated for uint64_t keys
// without payloads.
#include "bcf_segmented.cuh"

namespace bcf {

template cudaError_t launch_segmented_kp<uint64_t, false>(int, const SegArgs&, cudaStream_t);

}  // namespace bcf
