// bcf_block_sort_u64.cu -- the block sort instantiated for 64-bit keys, with and without payloads.
#include "bcf_block_sort.cuh"

namespace bcf {

template cudaError_t launch_block_sort_typed<uint64_t, false>(int, const BlockSortArgs&,
                                                              cudaStream_t);
template cudaError_t launch_block_sort_typed<uint64_t, true>(int, const BlockSortArgs&,
                                                             cudaStream_t);

}  // namespace bcf
