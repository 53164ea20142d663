// bcf_block_sort.cu -- dispatch of the base-case block sort (the kernel is in
// bcf_block_sort.cuh, instantiated per key type in bcf_block_sort_*.cu).
#include <cuda_runtime.h>

#include "bcf_internal.h"

namespace bcf {

template <typename K, bool PAIRS>
cudaError_t launch_block_sort_typed(int cfg, const BlockSortArgs& a, cudaStream_t s);

// Register budget: 64-bit keys with payloads carry four words per element,
// so only E = 16 is built for them.  Every other kind also has E = 32 tiles
// (u32 pairs: 128 registers, 64-bit keys: 80, no spills): tiles two to four
// times larger than E = 16 allows, so one or two merge passes fewer.
bool block_cfg_supported(int key_bytes, bool pairs, int cfg) {
  if (cfg < 0 || cfg >= kNumBlockCfgs) return false;
  if (key_bytes != 4 && key_bytes != 8) return false;
  if (pairs && key_bytes == 8) return kBlockCfgs[cfg].E == 16;
  if (kBlockCfgs[cfg].NT > 512) return !pairs && key_bytes == 4;
  return true;
}

cudaError_t launch_block_sort(int key_bytes, bool pairs, int cfg, const BlockSortArgs& a,
                              cudaStream_t s) {
  if (!block_cfg_supported(key_bytes, pairs, cfg)) return cudaErrorInvalidValue;
  if (key_bytes == 4)
    return pairs ? launch_block_sort_typed<uint32_t, true>(cfg, a, s)
                 : launch_block_sort_typed<uint32_t, false>(cfg, a, s);
  return pairs ? launch_block_sort_typed<uint64_t, true>(cfg, a, s)
               : launch_block_sort_typed<uint64_t, false>(cfg, a, s);
}

}  // namespace bcf
