// bcf_block_sort_u32p.cu -- the block sort instantiated for 32-bit keys with u32 payloads.
#include "bcf_block_sort.cuh"

namespace bcf {

template cudaError_t launch_block_sort_typed<uint32_t, true>(int, const BlockSortArgs&, cudaStream_t);

}  // namespace bcf
