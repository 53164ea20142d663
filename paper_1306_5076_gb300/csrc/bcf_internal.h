// bcf_internal.h -- launch interface between the C-ABI host code and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace bcf {

// Library-wide run-time settings (bcf_api.cu).  wait_limit_ns(): the limit of
// every device-side bounded wait (bcf_set_wait_limit_us); the launch wrappers
// copy it into their kernels' arguments.  smem_floor_bytes(): the profiling
// floor on the block sort's and merge pass's dynamic shared memory
// (bcf_profile_set_smem_floor); 0 leaves every launch as built.
uint64_t wait_limit_ns();
uint32_t smem_floor_bytes();
// chained_launches(): false while the launch profiler is on, whose events
// between launches must see each kernel start after its predecessor ended.
bool chained_launches();
constexpr uint64_t kDefaultWaitLimitNs = 2000000000ull;  // 2 s
constexpr uint32_t kMaxWaitLimitUs = 60000000u;          // 60 s
constexpr uint32_t kMaxSmemFloor = 227u * 1024u;         // the opt-in maximum per CTA

// Launch of a kernel that begins with pdl_wait() (bcf_device.cuh) as a
// programmatic dependent of the kernel ahead of it in the stream: it is
// scheduled once that kernel's last CTA has run, and starts work once that
// kernel has completed.  Only kernels whose every global access follows
// pdl_wait() may be launched this way.  While the launch profiler is on, a
// plain launch.
template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                           cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = chained_launches() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

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
// samples first and then only inside a window of +-kSampleStride keys.  The
// window's probes are the partition's DRAM reads (the samples stay cached):
// measured at 2^28 u32 keys, 64 takes the partition from 40 to 29 us per
// pass (the sort 7.05 -> 6.90 ms) for 1.6 % more sample writes.
constexpr uint32_t kSampleStride = 64;
// Merges of given runs (bcf_merge_runs) sample their input with a kernel of
// its own, reading one sector per sample: there a 256-key stride keeps that
// read at 3 % of the data (64 keys cost 12 % and took the one-pass merge of
// two runs from 0.21 to 0.24 ms).  The workspace's sample arrays are sized
// for the smaller stride.
constexpr uint32_t kRunSampleStride = 256;
static_assert(kRunSampleStride % kSampleStride == 0, "sample arrays sized by kSampleStride");

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
  uint32_t run_log2;    // regular mode: log2 L (L is a power of two)
  uint64_t* splits;     // per work item: A-split at the item's first output diagonal
  int mode_in;
  int mode_out;
  uint32_t* err;        // device error word
  uint64_t nitems;      // work items (tile pieces) of this launch
  const void* samples_in;  // sample array of kin (key g / S at every g = 0 mod S), or nullptr
  void* samples_out;       // sample array of kout, or nullptr
  uint64_t wait_ns;        // bounded-wait limit (set by launch_merge)
};

// Tuning configuration: elements per thread and threads per CTA.
struct TileCfg {
  int E, NT;
  constexpr int tile() const { return E * NT; }
};

// Supported configurations (index into these tables).
// E is 16 or 32 and the tile E*NT lies in [2^10, E^3], the range the three
// register layouts of bcf_device.cuh cover.  Block tiles {4096, 8192, 16384,
// 4096, 32768}; merge tiles {4096, 4096, 8192, 2048}.  The 32768-key block
// tile (1024 threads, 135 KB of shared memory, one CTA per SM) is built for
// 32-bit keys without payloads only: it saves a merge pass for 15 more
// network stages per key.
constexpr TileCfg kBlockCfgs[] = {{16, 256}, {32, 256}, {32, 512}, {32, 128}, {32, 1024}};
constexpr TileCfg kMergeCfgs[] = {{16, 256}, {32, 128}, {32, 256}, {16, 128}};
constexpr int kNumBlockCfgs = sizeof(kBlockCfgs) / sizeof(kBlockCfgs[0]);
constexpr int kNumMergeCfgs = sizeof(kMergeCfgs) / sizeof(kMergeCfgs[0]);

// Is the configuration compiled for this key width / payload flag?
bool block_cfg_supported(int key_bytes, bool pairs, int cfg);
bool merge_cfg_supported(int key_bytes, bool pairs, int cfg);

// ---------------------------------------------------------------- sort workspace

constexpr int ilog2_u64(uint64_t x) { return x <= 1 ? 0 : 1 + ilog2_u64(x >> 1); }

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Smallest merge tile over all configurations: bounds the split arrays.
constexpr uint64_t kMinMergeTile = 2048;
constexpr bool merge_tiles_at_least(uint64_t t) {
  for (int i = 0; i < kNumMergeCfgs; ++i)
    if (static_cast<uint64_t>(kMergeCfgs[i].tile()) < t) return false;
  return true;
}
static_assert(merge_tiles_at_least(kMinMergeTile), "a merge tile is below kMinMergeTile");

struct WsLayout {
  size_t splits, samples0, samples1, keys, vals, total;
};

// Workspace of a sort or a merge of runs_or_segs runs:
// [header | splits | samples of the output buffer | samples of the workspace
// copy | keys copy | values copy].  constexpr so that fixed-size scratch
// (bcf_static.cu) is sized by the same formula at compile time.
constexpr WsLayout ws_layout(uint64_t n, uint64_t runs_or_segs, int kb, bool pairs) {
  WsLayout w{};
  const uint64_t items = (n + kMinMergeTile - 1) / kMinMergeTile + runs_or_segs + 2;
  const uint64_t nsamp = n / kSampleStride + 2;
  w.splits = kAlign;
  w.samples0 = align_up(w.splits + items * sizeof(uint64_t), kAlign);
  w.samples1 = align_up(w.samples0 + nsamp * kb, kAlign);
  w.keys = align_up(w.samples1 + nsamp * kb, kAlign);
  w.vals = align_up(w.keys + n * kb, kAlign);
  w.total = align_up(w.vals + (pairs ? n * 4 : 0), kAlign);
  return w;
}

// Segmented sort (persistent kernel); tile = merge tile = E * NT.
constexpr TileCfg kSegCfgs[] = {{16, 256}, {16, 128}, {32, 128}, {32, 256}, {32, 512}};
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
  int skip_odd;          // leave odd-indexed segments untouched (pivot buckets)
  void* queue;           // work descriptors, `capacity` of them, cleared to 0
  uint64_t capacity;
  uint32_t* items_left;  // nseg
  uint32_t* tiny_list;   // nseg
  uint64_t* tile_base;   // nseg: index of the segment's first tile among all segments' tiles
  uint64_t* piece_split; // one per tile of all segments: merge-path split of its next piece
  void* ctl;             // queue counters
  uint32_t* err;
  // Merge passes outside the worker (merge_cfg >= 0): segments of two or more
  // tiles are only block-sorted by the worker; their merge passes run as
  // launches of the merge kernel over a device list (SegPassList).
  int merge_cfg;           // -1: the worker merges; else the merge kernel configuration
  uint32_t* order;         // nseg: multi-tile segments, most passes first
  uint64_t* piece_end;     // nseg: inclusive prefix sums of their merge tiles in that order
  uint32_t* count_ge;      // kSegMaxPasses + 2: count_ge[q] = listed segments with >= q passes
  void* samples_out;       // keys at positions that are multiples of kRunSampleStride in
  void* samples_buf;       // the output / in the workspace copy (listed segments)
};
bool seg_cfg_supported(int key_bytes, bool pairs, int cfg);
cudaError_t launch_segmented(int key_bytes, bool pairs, int cfg, const SegLaunch& L,
                             cudaStream_t s);
size_t seg_work_bytes();
// One CTA of the 32-bit worker on a queue whose only announced slot is never
// published: its bounded wait runs out (failure-path self-test).  ws: at
// least kSegSelftestBytes of device memory, 256-byte aligned.
constexpr size_t kSegSelftestBytes = 512;
cudaError_t launch_segmented_wait_selftest(void* ws, uint64_t wait_ns, uint32_t* err,
                                           cudaStream_t s);
size_t seg_ctl_bytes();

cudaError_t launch_block_sort(int key_bytes, bool pairs, int cfg, const BlockSortArgs& a,
                              cudaStream_t s);
cudaError_t launch_partition(int key_bytes, int cfg, const MergeArgs& a, const PairList* pl,
                             cudaStream_t s);
// Samples of keys [lo, hi): samples[g / kRunSampleStride] = (mapped) keys[g]
// for every g in [lo, hi) that is a multiple of kRunSampleStride (merges of
// given runs).
cudaError_t launch_sample_span(int key_bytes, const void* keys, void* samples, int mode,
                               uint64_t lo, uint64_t hi, cudaStream_t s);
cudaError_t launch_merge(int key_bytes, bool pairs, int cfg, const MergeArgs& a,
                         const PairList* pl, cudaStream_t s);

// Merge passes of a segmented sort's multi-tile segments, outside the worker.
// Segment s, block-sorted in tiles of T keys (T-aligned, clipped to the
// segment), needs P_s = ceil(log2 tiles) pairwise passes; its pass j merges
// runs of 2^(j-1) tiles.  The list holds the segments with P_s >= 1, most
// passes first, so the segments that still have q or more passes to go are
// a prefix of it; one launch does, for every one of those, the pass that
// leaves q - 1 to go (its pass P_s - q + 1).  All of them read the same
// buffer and write the same one in that launch.  Work items are the
// Tm-aligned output tiles of the listed segments (Tm divides T, so an item
// lies in one pair); the partition writes each item's pair and split, the
// merge kernel reads them.
constexpr uint32_t kSegMaxPasses = 40;
struct SegItem {
  uint64_t src, na, nb, out0;  // pair A = [src, src + na), B = next nb; tile start
};
struct SegPassList {
  const uint64_t* off;
  const uint32_t* order;
  const uint64_t* piece_end;
  const uint32_t* count_ge;
  SegItem* items;
  uint32_t* chunk_seg;         // list position of work item 32 c (launch_seg_chunks)
  unsigned long long* next;    // per q: work items taken by the merge launch's CTAs
  uint64_t n;
  uint32_t T;   // block-sort tile of the segmented sort
  uint32_t q;   // passes to go, this one included
};
// Once per sort, before its merge launches: the chunk table of the list (the
// list position of every 32nd work item) and the merge launches' counters.
cudaError_t launch_seg_chunks(const SegPassList& L, cudaStream_t s);
cudaError_t launch_seg_partition(int key_bytes, int cfg, const MergeArgs& a,
                                 const SegPassList& L, cudaStream_t s);
cudaError_t launch_seg_merge(int key_bytes, bool pairs, int cfg, const MergeArgs& a,
                             const SegPassList& L, cudaStream_t s);

// Colored prefix sums (Appendix A).  One tile of kCpsTile elements per CTA,
// tiles taken in order from `counter`; `status` holds one word per (tile,
// color) for the look-back across tiles and must be zero before the launch.
constexpr int kCpsThreads = 256;
constexpr int kCpsPerThread = 16;  // elements per thread and step
constexpr int kCpsSteps = 4;       // steps per tile: each thread owns 64 consecutive elements
constexpr int kCpsTile = kCpsThreads * kCpsPerThread * kCpsSteps;
constexpr uint32_t kCpsMaxColors = 64;
constexpr uint32_t kErrBadColor = 8u;          // device error bit: a color >= d
constexpr uint32_t kErrLookbackTimeout = 16u;  // device error bit: look-back wait ran out
constexpr uint32_t kErrSelftestTimeout = 32u;  // device error bit: the self-test's wait ran out
struct CpsArgs {
  uint32_t* out;
  const uint32_t* values;
  const uint8_t* colors;  // nullptr: every element has color 0 (a plain scan, d = 1)
  uint64_t n;
  uint32_t d;            // colors, 1..kCpsMaxColors
  int exclusive;
  uint64_t ntiles;
  unsigned long long* status;  // ntiles * d words
  uint32_t* counter;     // next tile
  uint32_t* err;
  uint64_t wait_ns;      // bounded-wait limit of the look-back (set by launch_cps)
};
// layout 0: one shared-memory bank per thread (the paper's conflict-free
// layout); layout 1: each thread's d counters contiguous (the conflicting one).
cudaError_t launch_cps(const CpsArgs& a, int layout, cudaStream_t s);
size_t cps_smem_bytes(uint32_t d);

// Pivot buckets (BCFMergesortPB, Sec. 3.2): P - 1 splitters from every
// kPbSampleStride-th key; buckets open(0), equal(s_0), open(1), ..., open(m).
constexpr uint32_t kPbSampleStride = 256;
constexpr uint32_t kPbP = 256;
constexpr uint32_t kPbSplitters = kPbP - 1;
constexpr uint32_t kPbBuckets = 2 * kPbSplitters + 1;
enum { kPbStepSample, kPbStepSplitters, kPbStepCount, kPbStepScatter, kPbStepSegOffsets,
       kPbStepEqualCount };
struct PbArgs {
  const void* kin;            // user keys (original bits)
  uint64_t n;
  int mode;                   // key map of the sort
  void* samples;              // ns mapped keys
  uint64_t ns;
  const void* sorted_samples; // the samples, sorted
  void* splitters;            // up to kPbSplitters mapped keys
  uint32_t* nsplit;           // m
  const void* x;              // block-sorted tiles (mapped keys)
  const uint32_t* xv;         // their payloads, or nullptr
  uint32_t T;                 // block tile
  uint64_t ntiles;
  uint32_t* counts;           // kPbBuckets * ntiles piece sizes, bucket-major
  const uint32_t* offsets;    // their exclusive prefix sum: piece output positions
  void* kout;                 // final output (original bits)
  uint32_t* vout;
  uint64_t* seg_off;          // kPbBuckets + 1 bucket boundaries
  uint32_t sample_stride;     // candidates are the keys at multiples of this (kPbSampleStride)
  uint32_t* equal_count;      // kPbStepEqualCount: sorted samples equal to a splitter (zeroed)
};
cudaError_t launch_pb(int step, int key_bytes, bool pairs, const PbArgs& a, cudaStream_t s);

// Conversions (bcf_convert.cu): 16-bit keys through the 32-bit sort, and wide
// payloads gathered by sorted row index.
cudaError_t launch_widen16(uint32_t* out, const uint16_t* in, uint64_t n, bool sign,
                           cudaStream_t s);
cudaError_t launch_narrow16(uint16_t* out, const uint32_t* in, uint64_t n, cudaStream_t s);
cudaError_t launch_iota(uint32_t* v, uint64_t n, cudaStream_t s);
cudaError_t launch_gather(void* out, const void* in, const uint32_t* idx, uint64_t n,
                          uint32_t row_bytes, cudaStream_t s);

}  // namespace bcf
