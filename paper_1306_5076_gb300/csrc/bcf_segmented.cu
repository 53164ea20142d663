// bcf_segmented.cu -- sorting many independent segments (the batching
// extension of the paper's method; the paper's own "segmented ShearSort"
// sorts segments inside one tile, Sec. 3.1 and Algorithm 5).
//
// Plan (plan_kernel, one CTA): every segment is classified --
//   tiny   : 1..512 keys, sorted by one warp entirely in registers (Batcher's
//            network per lane, then bitonic merges across lanes by shuffle);
//   others : block-sorted in T-key tiles (T-aligned in the array, clipped to
//            the segment, ragged ends padded), then merged pairwise with
//            ceil(log2 tiles) segment-local merge passes (Sec. 3.2; Lemma 2).
// The plan queues groups of tiny segments (one per warp of a worker CTA);
// fill_tiles_kernel queues the tile sorts, one thread per slot.
//
// The merge passes run in one of two forms, chosen by the tuning table:
//
// 1. In the persistent worker (seg_worker, one wave of co-resident CTAs):
// each CTA repeatedly takes the next queue slot.  When the last item of a
// segment's pass completes, the CTA that completed it enqueues the segment's
// next pass (one item per T-aligned output tile of the segment), so every
// segment advances as soon as its own data is ready and no grid-wide barrier
// exists.  Waiting for a slot to be published is bounded (global timer); on
// expiry the device error word is set and the CTA exits.  The CTA that
// publishes a segment's merge pass first finds the exact splitters of all its
// pieces (merge path, one warp per piece, 32-ary search), so a piece starts
// with its two splits in hand -- for passes of up to 16 pieces per warp; a
// longer segment's pieces search their own, so that one huge segment does not
// wait on a single CTA.  Pieces read their windows straight from global
// memory (.cg loads: data written by other SMs earlier in the same launch
// must not be served from a stale L1 line), then run the same conflict-free
// bitonic merge as the merge pass kernel.
//
// 2. As launches of the merge kernel (bcf_seg_merge.cu): the plan also lists
// the segments of two or more tiles, most passes first; the tile sorts run
// one CTA per tile (seg_tile_kernel) and the tiny segments one warp each
// (seg_tiny_kernel); the host then launches a partition and a merge per
// number of passes to go.
#include <cuda_runtime.h>

#include "bcf_segmented.cuh"

namespace bcf {

// ---------------------------------------------------------------- plan

// Inclusive block scan of one value per thread (blockDim.x == 1024).
template <typename T>
__device__ __forceinline__ T block_scan_incl(T v, T* warp_sums, T& total) {
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T u = __shfl_up_sync(0xFFFFFFFFu, v, d);
    if (lane >= static_cast<uint32_t>(d)) v += u;
  }
  if (lane == 31) warp_sums[w] = v;
  __syncthreads();
  if (w == 0) {
    T x = warp_sums[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const T u = __shfl_up_sync(0xFFFFFFFFu, x, d);
      if (lane >= static_cast<uint32_t>(d)) x += u;
    }
    warp_sums[lane] = x;
  }
  __syncthreads();
  if (w > 0) v += warp_sums[w - 1];
  total = warp_sums[31];
  __syncthreads();
  return v;
}

// Inclusive block scan of three values per thread at once (blockDim.x ==
// 1024): one set of barriers for the plan's three running sums.
__device__ __forceinline__ void block_scan3_incl(unsigned long long (&v)[3],
                                                 unsigned long long (*warp_sums)[32],
                                                 unsigned long long (&total)[3]) {
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, v[i], d);
      if (lane >= static_cast<uint32_t>(d)) v[i] += u;
    }
  }
  if (lane == 31) {
#pragma unroll
    for (int i = 0; i < 3; ++i) warp_sums[i][w] = v[i];
  }
  __syncthreads();
  if (w < 3) {  // warp i scans the warp sums of value i
    unsigned long long x = warp_sums[w][lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, x, d);
      if (lane >= static_cast<uint32_t>(d)) x += u;
    }
    warp_sums[w][lane] = x;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (w > 0) v[i] += warp_sums[i][w - 1];
    total[i] = warp_sums[i][31];
  }
  __syncthreads();
}

// The list of segments whose merge passes run outside the worker: a counting
// sort by pass count (most passes first; within a count, in no particular
// order), then the inclusive prefix sums of their Tm-tiles in list order.
// hist[P] holds the number of listed segments with P passes.
__device__ __forceinline__ void plan_list(const SegArgs& a, uint32_t T, uint32_t* hist) {
  __shared__ unsigned long long ws[32];
  __shared__ uint32_t cursor[kSegMaxPasses + 2];
  __syncthreads();  // every count is in hist
  if (threadIdx.x == 0) {
    uint32_t ge = 0;
    a.count_ge[kSegMaxPasses + 1] = 0;
    for (int q = kSegMaxPasses; q >= 0; --q) {
      cursor[q] = ge;  // the segments with more passes come first
      ge += q > 0 ? hist[q] : 0u;
      a.count_ge[q] = ge;
    }
  }
  __syncthreads();
  for (uint64_t s = threadIdx.x; s < a.nseg; s += blockDim.x) {
    const SegGeo g = seg_geo(a.off, s, a.n, T, a.skip_odd != 0);
    if (g.passes == 0) continue;
    const uint32_t pos =
        atomicAdd(&cursor[g.passes < kSegMaxPasses ? g.passes : kSegMaxPasses], 1u);
    a.order[pos] = static_cast<uint32_t>(s);
    a.piece_end[pos] = (g.hi - 1) / a.Tm - g.lo / a.Tm + 1;
  }
  __syncthreads();
  const uint32_t listed = a.count_ge[1];
  unsigned long long carry = 0;
  for (uint32_t c = 0; c < listed; c += blockDim.x) {
    const uint32_t i = c + threadIdx.x;
    const unsigned long long v = i < listed ? a.piece_end[i] : 0ull;
    unsigned long long sum;
    const unsigned long long incl = block_scan_incl(v, ws, sum);
    if (i < listed) a.piece_end[i] = carry + incl;
    carry += sum;
  }
}

__global__ void __launch_bounds__(1024) plan_kernel(const SegArgs a, uint32_t T,
                                                    uint32_t per_group) {
  __shared__ unsigned long long ws[3][32];
  __shared__ uint32_t s_hist[kSegMaxPasses + 2];
  for (uint32_t q = threadIdx.x; q < kSegMaxPasses + 2; q += blockDim.x) s_hist[q] = 0;
  __syncthreads();
  const bool defer = a.Tm != 0;
  unsigned long long carry_tiles = 0, carry_tiny = 0, carry_total = 0;
  for (uint64_t c = 0; c < a.nseg; c += 1024) {
    const uint64_t s = c + threadIdx.x;
    SegGeo g{};
    if (s < a.nseg) g = seg_geo(a.off, s, a.n, T, a.skip_odd != 0);
    const unsigned long long tiles = g.tiles;
    const unsigned long long tiny = g.tiny ? 1 : 0;
    // a listed segment's merge passes are not queue items
    const bool listed = defer && g.passes > 0;
    const unsigned long long tot =
        tiles + (listed ? 0ull : static_cast<unsigned long long>(g.passes) * g.pieces);
    if (listed) atomicAdd(&s_hist[g.passes < kSegMaxPasses ? g.passes : kSegMaxPasses], 1u);
    unsigned long long v[3] = {tiles, tiny, tot}, sum[3];
    block_scan3_incl(v, ws, sum);
    const unsigned long long t_excl = v[0] - tiles;
    const unsigned long long y_incl = v[1];
    const unsigned long long sum_tiles = sum[0], sum_tiny = sum[1], sum_tot = sum[2];
    if (s < a.nseg) {
      a.items_left[s] = g.tiles;
      a.tile_base[s] = carry_tiles + t_excl;
      if (g.tiny) a.tiny_list[carry_tiny + y_incl - 1] = static_cast<uint32_t>(s);
    }
    carry_tiles += sum_tiles;
    carry_tiny += sum_tiny;
    carry_total += sum_tot;
  }
  const unsigned long long groups = (carry_tiny + per_group - 1) / per_group;
  for (unsigned long long q = threadIdx.x; q < groups; q += blockDim.x) {
    if (carry_tiles + q < a.capacity) {
      SegWork w;
      w.meta = kReady | kWTiny;
      w.seg = 0;
      w.arg = q;
      a.queue[carry_tiles + q] = w;
    }
  }
  if (defer) plan_list(a, T, s_hist);
  if (threadIdx.x == 0) {
    const unsigned long long total = carry_total + groups;
    a.ctl->head = 0;
    a.ctl->reserve = carry_tiles + groups;
    a.ctl->total = total <= a.capacity ? total : 0;  // overflow: nothing runs
    a.ctl->n_tiny = carry_tiny;
    a.ctl->tiles = total <= a.capacity ? carry_tiles : 0;
    if (total > a.capacity) atomicOr(a.err, kErrQueueOverflow);
  }
}

// The tile-sort slots [0, tiles) of the queue, in parallel: slot idx belongs
// to the last segment whose first tile index (tile_base, non-decreasing) is
// at most idx.  (A single thread per segment would write a segment of 2^31
// keys' 2^19 slots alone.)
__global__ void __launch_bounds__(256) fill_tiles_kernel(const SegArgs a) {
  const uint64_t tiles = __ldcg(&a.ctl->tiles);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t idx = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
       idx < tiles; idx += stride) {
    uint64_t lo = 0, hi = a.nseg;  // first segment whose tile_base exceeds idx
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (__ldcg(a.tile_base + mid) > idx) hi = mid; else lo = mid + 1;
    }
    const uint64_t s = lo - 1;
    SegWork w;
    w.meta = kReady | kWTile;
    w.seg = static_cast<uint32_t>(s);
    w.arg = idx - __ldcg(a.tile_base + s);
    a.queue[idx] = w;
  }
}

cudaError_t launch_plan(const SegArgs& a, uint32_t T, uint32_t tiny_per_group, cudaStream_t s) {
  plan_kernel<<<1, 1024, 0, s>>>(a, T, tiny_per_group);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // a segment touches at most size / T + 2 tiles
  const uint64_t bound = a.n / T + 2 * a.nseg + 2;
  const uint64_t blocks = (bound + 255) / 256;
  fill_tiles_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- host side

bool seg_cfg_supported(int key_bytes, bool pairs, int cfg) {
  if (cfg < 0 || cfg >= kNumSegCfgs) return false;
  if (key_bytes != 4 && key_bytes != 8) return false;
  return kSegCfgs[cfg].E == 16 || (!pairs && key_bytes == 4);
}

cudaError_t launch_segmented(int key_bytes, bool pairs, int cfg, const SegLaunch& L,
                             cudaStream_t s) {
  if (!seg_cfg_supported(key_bytes, pairs, cfg)) return cudaErrorInvalidValue;
  SegArgs a;
  a.kin = L.kin;
  a.vin = L.vin;
  a.kout = L.kout;
  a.vout = L.vout;
  a.kbuf = L.kbuf;
  a.vbuf = L.vbuf;
  a.off = L.off;
  a.nseg = L.nseg;
  a.n = L.n;
  a.mode = L.mode;
  a.skip_odd = L.skip_odd;
  a.queue = static_cast<SegWork*>(L.queue);
  a.capacity = L.capacity;
  a.items_left = L.items_left;
  a.tiny_list = L.tiny_list;
  a.tile_base = L.tile_base;
  a.piece_split = L.piece_split;
  a.ctl = static_cast<SegCtl*>(L.ctl);
  a.err = L.err;
  a.wait_ns = wait_limit_ns();
  a.Tm = L.merge_cfg >= 0 ? static_cast<uint32_t>(kMergeCfgs[L.merge_cfg].tile()) : 0u;
  a.order = L.order;
  a.piece_end = L.piece_end;
  a.count_ge = L.count_ge;
  a.samples_out = a.Tm ? L.samples_out : nullptr;
  a.samples_buf = a.Tm ? L.samples_buf : nullptr;
  if (key_bytes == 4)
    return pairs ? launch_segmented_kp<uint32_t, true>(cfg, a, s)
                 : launch_segmented_kp<uint32_t, false>(cfg, a, s);
  return pairs ? launch_segmented_kp<uint64_t, true>(cfg, a, s)
               : launch_segmented_kp<uint64_t, false>(cfg, a, s);
}

size_t seg_work_bytes() { return sizeof(SegWork); }
size_t seg_ctl_bytes() { return sizeof(SegCtl); }

}  // namespace bcf
