// bcf_internal.h -- launch interface between the C-ABI host code and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace bcf {

// One adjacent pair of sorted runs to merge: A = [off, off + na), B = [off + na,
// off + na + nb) of the source array; the merged run occupies the same index
// range of the destination.  `piece0` is the index of the pair's first work
// item (tile piece); the pair has pieces covering the Tm-aligned output tiles
// its range touches.
struct PairDesc {
  uint64_t off, na, nb, piece0;
};

// Maximum pairs passed by value to one irregular merge launch.
constexpr int kMaxPairsPerLaunch = 256;

struct PairList {
  PairDesc p[kMaxPairsPerLaunch];
  uint32_t npairs;
  uint32_t pad_;
};

// Every kSampleStride-th key of each sorted run is also written to a sample
// array (in mapped key order); the next pass's merge-path search runs on the
// samples first and then only inside a window of +-kSampleStride keys.
constexpr uint32_t kSampleStride = 256;

struct BlockSortArgs {
  const void* kin;
  const uint32_t* vin;  // nullptr for keys only
  void* kout;
  uint32_t* vout;
  uint64_t n;           // elements of the array
  int mode_in;          // key map applied on load (bit0 f32 order, bit1 descending)
  int mode_out;         // inverse key map applied on store
  void* samples;        // sample array of kout (keys at multiples of kSampleStride), or nullptr
};

struct MergeArgs {
  const void* kin;
  const uint32_t* vin;
  void* kout;
  uint32_t* vout;
  uint64_t n;           // regular mode: elements of the array
  uint64_t run;         // regular mode: run length L (pairs of runs are 2L apart)
  uint64_t* splits;     // per work item: A-split at the item's first output diagonal
  int mode_in;
  int mode_out;
  uint32_t* err;        // device error word
  uint64_t nitems;      // work items (tile pieces) of this launch
  const void* samples_in;  // regular mode: sample array of kin, or nullptr
  void* samples_out;       // regular mode: sample array of kout, or nullptr
};

// Tuning configuration: elements per thread and threads per CTA.
struct TileCfg {
  int E, NT;
  constexpr int tile() const { return E * NT; }
};

// Supported configurations (index into these tables).
// E is 16 or 32 and the tile E*NT lies in [2^10, E^3], the range the three
// register layouts of bcf_device.cuh cover.  Block tiles {4096, 8192, 16384,
// 4096}; merge tiles {4096, 4096, 8192, 2048}.
constexpr TileCfg kBlockCfgs[] = {{16, 256}, {32, 256}, {32, 512}, {32, 128}};
constexpr TileCfg kMergeCfgs[] = {{16, 256}, {32, 128}, {32, 256}, {16, 128}};
constexpr int kNumBlockCfgs = sizeof(kBlockCfgs) / sizeof(kBlockCfgs[0]);
constexpr int kNumMergeCfgs = sizeof(kMergeCfgs) / sizeof(kMergeCfgs[0]);

// Is the configuration compiled for this key width / payload flag?
bool block_cfg_supported(int key_bytes, bool pairs, int cfg);
bool merge_cfg_supported(int key_bytes, bool pairs, int cfg);

// Segmented sort (persistent kernel); tile = merge tile = E * NT.
constexpr TileCfg kSegCfgs[] = {{16, 256}, {16, 128}, {32, 128}};
constexpr int kNumSegCfgs = sizeof(kSegCfgs) / sizeof(kSegCfgs[0]);
constexpr uint64_t kMinSegTile = 2048;

struct SegLaunch {
  const void* kin;
  const uint32_t* vin;
  void* kout;
  uint32_t* vout;
  void* kbuf;            // workspace copy of the keys (ping-pong)
  uint32_t* vbuf;
  const uint64_t* off;   // device, nseg + 1
  uint64_t nseg, n;
  int mode;
  void* queue;           // work descriptors, `capacity` of them, cleared to 0
  uint64_t capacity;
  uint32_t* items_left;  // nseg
  uint32_t* tiny_list;   // nseg
  void* ctl;             // queue counters
  uint32_t* err;
};
bool seg_cfg_supported(int key_bytes, bool pairs, int cfg);
cudaError_t launch_segmented(int key_bytes, bool pairs, int cfg, const SegLaunch& L,
                             cudaStream_t s);
size_t seg_work_bytes();
size_t seg_ctl_bytes();

cudaError_t launch_block_sort(int key_bytes, bool pairs, int cfg, const BlockSortArgs& a,
                              cudaStream_t s);
cudaError_t launch_partition(int key_bytes, int cfg, const MergeArgs& a, const PairList* pl,
                             cudaStream_t s);
cudaError_t launch_merge(int key_bytes, bool pairs, int cfg, const MergeArgs& a,
                         const PairList* pl, cudaStream_t s);

}  // namespace bcf
