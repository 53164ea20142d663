// bcf_segmented_u32m.cu -- the persistent segmented sort instantiated for uint32_t keys
// without payloads whose order is mapped (f32 totalOrder, i32, descending).
#include "bcf_segmented.cuh"

namespace bcf {

template cudaError_t dispatch_seg<uint32_t, false, true>(int, const SegArgs&, cudaStream_t);

}  // namespace bcf
