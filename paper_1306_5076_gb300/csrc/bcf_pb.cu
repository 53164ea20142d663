// bcf_pb.cu -- pivot buckets: the distribution step of BCFMergesortPB
// (Sec. 3.2, paragraphs "Distribution" and "Duplicate keys").
//
// The paper stops merging when the number of sorted sequences reaches the
// number of processors P, picks t evenly spaced elements of every sequence as
// candidate splitters, sorts them, keeps P - 1 evenly spaced ones, ranks every
// splitter in every sequence, moves every piece to its bucket, and merges the
// pieces of each bucket.  The PB variant gives the keys equal to a splitter
// buckets of their own: those are in final position once distributed, so
// duplicate-heavy inputs skip most of the remaining work.
//
// On GB300 (host sequence in bcf_api.cu, run_sort_pb):
//   1. pb_sample_kernel: every 256th input key (mapped to unsigned order)
//      is a candidate splitter; the candidates are sorted with the library's
//      own sort;
//   2. pb_splitter_kernel: P - 1 = 255 evenly spaced candidates, duplicates
//      dropped, give m <= 255 strictly increasing splitters and the bucket
//      order open(0), equal(s_0), open(1), equal(s_1), ..., open(m);
//   3. the block sort sorts the input in T-key tiles (the sequences);
//   4. pb_count_kernel: one CTA per tile ranks every splitter in the tile
//      (lower and upper bound, binary searches in shared memory) and writes
//      the tile's piece size for every bucket, bucket-major;
//   5. an exclusive prefix sum of the piece sizes (the colored prefix sum
//      kernel with one color) gives every piece its output position;
//   6. pb_scatter_kernel: every tile moves its pieces there (keys unmapped,
//      payloads along), so each equal bucket is final and stable (pieces in
//      tile order, each in input order);
//   7. the segmented sort, in place, sorts the open buckets only (odd,
//      equal buckets are skipped).
// Step 7 sorts each open bucket's pieces afresh instead of merging them
// (the pieces are sorted; the segmented sort does not use that).
#include <cuda_runtime.h>

#include "bcf_device.cuh"
#include "bcf_internal.h"

namespace bcf {

namespace {

constexpr int kPbThreads = 256;

template <typename K, bool MAP>
__global__ void pb_sample_kernel(const PbArgs a) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.ns) return;
  const K x = static_cast<const K*>(a.kin)[i * a.sample_stride];
  static_cast<K*>(a.samples)[i] = MAP ? map_key(x, a.mode) : x;
}

// One CTA of kPbThreads threads: candidate j < P - 1 is the sorted sample at
// rank (j + 1) * ns / P; a candidate equal to the previous one is dropped.
// The candidates are taken kPbThreads at a time, compacted in order.
template <typename K>
__global__ void __launch_bounds__(kPbThreads) pb_splitter_kernel(const PbArgs a) {
  __shared__ uint32_t warp_sums[kPbThreads / 32];
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const K* S = static_cast<const K*>(a.sorted_samples);
  uint32_t carry = 0;
  for (uint32_t j0 = 0; j0 < kPbSplitters; j0 += kPbThreads) {
    const uint32_t j = j0 + threadIdx.x;
    bool keep = false;
    K cand = 0;
    if (j < kPbSplitters) {
      cand = S[((j + 1) * a.ns) / kPbP];
      keep = j == 0 || cand != S[(j * a.ns) / kPbP];
    }
    // exclusive block scan of the keep flags
    const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, keep);
    const uint32_t before = __popc(ballot & ((1u << lane) - 1u));
    if (lane == 0) warp_sums[w] = __popc(ballot);
    __syncthreads();
    uint32_t base = carry, total = 0;
    for (uint32_t q = 0; q < kPbThreads / 32; ++q) {
      if (q < w) base += warp_sums[q];
      total += warp_sums[q];
    }
    if (keep) static_cast<K*>(a.splitters)[base + before] = cand;
    carry += total;
    __syncthreads();  // warp_sums is reused by the next chunk
  }
  if (threadIdx.x == 0) *a.nsplit = carry;
}

template <typename K>
__device__ __forceinline__ uint32_t lower_bound_sm(const K* x, uint32_t lo, uint32_t hi, K v) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (x[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
template <typename K>
__device__ __forceinline__ uint32_t upper_bound_sm(const K* x, uint32_t lo, uint32_t hi, K v) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (x[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Piece size of bucket b in a tile of `cnt` keys from the splitters' bounds.
__device__ __forceinline__ uint32_t bucket_size(uint32_t b, uint32_t m, const uint32_t* lo,
                                                const uint32_t* hi, uint32_t cnt) {
  if (b > 2 * m) return 0u;
  const uint32_t j = b >> 1;
  if (b & 1u) return hi[j] - lo[j];           // keys equal to splitter j
  const uint32_t start = j == 0 ? 0u : hi[j - 1];
  const uint32_t end = j < m ? lo[j] : cnt;  // keys between splitters j - 1 and j
  return end - start;
}

// One CTA per block-sorted tile.
template <typename K>
__global__ void __launch_bounds__(kPbThreads) pb_count_kernel(const PbArgs a) {
  extern __shared__ __align__(16) unsigned char pb_sm[];
  K* sk = reinterpret_cast<K*>(pb_sm);
  __shared__ uint32_t s_lo[kPbSplitters], s_hi[kPbSplitters];
  const uint64_t tile = blockIdx.x;
  const uint64_t base = tile * a.T;
  const uint64_t rem = a.n - base;
  const uint32_t cnt = rem < a.T ? static_cast<uint32_t>(rem) : a.T;
  const K* x = static_cast<const K*>(a.x) + base;
  for (uint32_t i = threadIdx.x; i < cnt; i += kPbThreads) sk[i] = x[i];
  const uint32_t m = *a.nsplit;
  __syncthreads();
  const K* sp = static_cast<const K*>(a.splitters);
  for (uint32_t j = threadIdx.x; j < m; j += kPbThreads) {
    const K v = sp[j];
    const uint32_t lo = lower_bound_sm(sk, 0u, cnt, v);
    s_lo[j] = lo;
    s_hi[j] = upper_bound_sm(sk, lo, cnt, v);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < kPbBuckets; b += kPbThreads)
    a.counts[static_cast<uint64_t>(b) * a.ntiles + tile] = bucket_size(b, m, s_lo, s_hi, cnt);
}

// One CTA per tile: every piece of the sorted tile (its slots of one bucket)
// is copied to its output position.  Pieces are cut into work items of
// kPbChunk slots, dealt to the warps in turn, so a few long pieces (duplicate
// keys) keep every warp busy; each lane keeps four loads in flight.
constexpr uint32_t kPbChunk = 1024;

template <typename K, bool PAIRS, bool MAP>
__global__ void __launch_bounds__(kPbThreads) pb_scatter_kernel(const PbArgs a) {
  __shared__ uint32_t s_start[kPbBuckets + 1];  // tile-local piece starts
  __shared__ uint32_t s_item[kPbBuckets + 1];   // first work item of each piece
  __shared__ uint32_t s_off[kPbBuckets];        // output position of each piece
  __shared__ uint32_t warp_sums[2][kPbThreads / 32];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
  const uint64_t tile = blockIdx.x;
  const uint64_t base = tile * a.T;
  const uint64_t rem = a.n - base;
  const uint32_t cnt = rem < a.T ? static_cast<uint32_t>(rem) : a.T;
  // exclusive scans over the buckets (two per thread) of the piece sizes and
  // of the work items per piece
  constexpr uint32_t kPer = (kPbBuckets + kPbThreads - 1) / kPbThreads;
  uint32_t c[kPer], sum = 0, items = 0;
#pragma unroll
  for (uint32_t q = 0; q < kPer; ++q) {
    const uint32_t b = tid * kPer + q;
    c[q] = b < kPbBuckets ? a.counts[static_cast<uint64_t>(b) * a.ntiles + tile] : 0u;
    if (b < kPbBuckets) s_off[b] = a.offsets[static_cast<uint64_t>(b) * a.ntiles + tile];
    sum += c[q];
    items += (c[q] + kPbChunk - 1) / kPbChunk;
  }
  uint32_t incl = sum, iincl = items;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    const uint32_t z = __shfl_up_sync(0xFFFFFFFFu, iincl, o);
    if (lane >= static_cast<uint32_t>(o)) {
      incl += y;
      iincl += z;
    }
  }
  if (lane == 31) {
    warp_sums[0][w] = incl;
    warp_sums[1][w] = iincl;
  }
  __syncthreads();
  uint32_t run = incl - sum, irun = iincl - items, total_items = 0;
  for (uint32_t q = 0; q < kPbThreads / 32; ++q) {
    if (q < w) {
      run += warp_sums[0][q];
      irun += warp_sums[1][q];
    }
    total_items += warp_sums[1][q];
  }
#pragma unroll
  for (uint32_t q = 0; q < kPer; ++q) {
    const uint32_t b = tid * kPer + q;
    if (b < kPbBuckets) {
      s_start[b] = run;
      s_item[b] = irun;
    }
    run += c[q];
    irun += (c[q] + kPbChunk - 1) / kPbChunk;
  }
  if (tid == 0) {
    s_start[kPbBuckets] = cnt;
    s_item[kPbBuckets] = total_items;
  }
  __syncthreads();
  const K* x = static_cast<const K*>(a.x) + base;
  const uint32_t* xv = PAIRS ? a.xv + base : nullptr;
  K* kout = static_cast<K*>(a.kout);
  for (uint32_t it = w; it < total_items; it += kPbThreads / 32) {
    // the piece of this item: last bucket whose first item is <= it (pieces
    // without items share their first item with the next piece)
    uint32_t lo = 0, hi = kPbBuckets + 1;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_item[mid] <= it) lo = mid; else hi = mid;
    }
    const uint32_t first = (it - s_item[lo]) * kPbChunk;
    const uint32_t len = s_start[lo + 1] - s_start[lo];
    const uint32_t stop = first + kPbChunk < len ? first + kPbChunk : len;
    const uint32_t src = s_start[lo];
    const uint64_t dst = s_off[lo];
    for (uint32_t i = first + lane; i < stop; i += 4 * 32) {
      K key[4];
      uint32_t val[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t j = i + u * 32;
        if (j < stop) {
          key[u] = x[src + j];
          if constexpr (PAIRS) val[u] = xv[src + j];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t j = i + u * 32;
        if (j < stop) {
          kout[dst + j] = MAP ? unmap_key(key[u], a.mode) : key[u];
          if constexpr (PAIRS) a.vout[dst + j] = val[u];
        }
      }
    }
  }
}

// How many sorted samples equal one of the m splitters (binary search of the
// splitters per sample): the share of keys that would land in equal buckets.
template <typename K>
__global__ void __launch_bounds__(kPbThreads) pb_equal_count_kernel(const PbArgs a) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  bool eq = false;
  if (i < a.ns) {
    const K v = static_cast<const K*>(a.sorted_samples)[i];
    const K* sp = static_cast<const K*>(a.splitters);
    uint32_t lo = 0, hi = *a.nsplit;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (sp[mid] < v) lo = mid + 1; else hi = mid;
    }
    eq = lo < *a.nsplit && sp[lo] == v;
  }
  const int cnt = __syncthreads_count(eq);
  if (threadIdx.x == 0 && cnt) atomicAdd(a.equal_count, static_cast<uint32_t>(cnt));
}

__global__ void pb_segoff_kernel(const PbArgs a) {
  for (uint32_t b = threadIdx.x; b < kPbBuckets; b += blockDim.x)
    a.seg_off[b] = a.offsets[static_cast<uint64_t>(b) * a.ntiles];  // tile 0's piece: bucket start
  if (threadIdx.x == 0) a.seg_off[kPbBuckets] = a.n;
}

template <typename K>
cudaError_t launch_pb_typed(int step, bool pairs, const PbArgs& a, cudaStream_t s) {
  const bool map = a.mode != 0;
  switch (step) {
    case kPbStepSample: {
      const unsigned grid = static_cast<unsigned>((a.ns + 255) / 256);
      if (map) pb_sample_kernel<K, true><<<grid, 256, 0, s>>>(a);
      else pb_sample_kernel<K, false><<<grid, 256, 0, s>>>(a);
      break;
    }
    case kPbStepSplitters:
      pb_splitter_kernel<K><<<1, kPbThreads, 0, s>>>(a);
      break;
    case kPbStepCount: {
      const size_t smem = static_cast<size_t>(a.T) * sizeof(K);
      cudaError_t err = cudaFuncSetAttribute(pb_count_kernel<K>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
      if (err != cudaSuccess) return err;
      pb_count_kernel<K><<<static_cast<unsigned>(a.ntiles), kPbThreads, smem, s>>>(a);
      break;
    }
    case kPbStepScatter: {
      const unsigned grid = static_cast<unsigned>(a.ntiles);
      if (pairs)
        map ? pb_scatter_kernel<K, true, true><<<grid, kPbThreads, 0, s>>>(a)
            : pb_scatter_kernel<K, true, false><<<grid, kPbThreads, 0, s>>>(a);
      else
        map ? pb_scatter_kernel<K, false, true><<<grid, kPbThreads, 0, s>>>(a)
            : pb_scatter_kernel<K, false, false><<<grid, kPbThreads, 0, s>>>(a);
      break;
    }
    case kPbStepSegOffsets:
      pb_segoff_kernel<<<1, 512, 0, s>>>(a);
      break;
    case kPbStepEqualCount: {
      const unsigned grid = static_cast<unsigned>((a.ns + kPbThreads - 1) / kPbThreads);
      pb_equal_count_kernel<K><<<grid, kPbThreads, 0, s>>>(a);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pb(int step, int key_bytes, bool pairs, const PbArgs& a, cudaStream_t s) {
  if (a.ntiles == 0 || a.ntiles > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  return key_bytes == 4 ? launch_pb_typed<uint32_t>(step, pairs, a, s)
                        : launch_pb_typed<uint64_t>(step, pairs, a, s);
}

}  // namespace bcf
