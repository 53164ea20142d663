// bcf_block_sort_u32k.cu -- the block sort instantiated for 32-bit keys without payloads.
#include "bcf_block_sort.cuh"

namespace bcf {

template cudaError_t launch_block_sort_typed<uint32_t, false>(int, const BlockSortArgs&, cudaStream_t);

}  // namespace bcf
