// bcf_seg_merge.cu -- the merge passes of a segmented sort's segments of two
// or more tiles, run as launches of the merge kernel over a device list
// instead of inside the persistent worker.  The worker block-sorts the tiles;
// the plan lists the segments with passes left, most passes first, with
// prefix sums of their merge tiles; one partition and one merge launch per
// number q of passes to go then do, for every listed segment with q or more
// passes left, its pass P_s - q + 1 (Sec. 3.2; Lemma 2 gives the pass count).
#include <cuda_runtime.h>

#include "bcf_merge.cuh"

namespace bcf {

// ---------------------------------------------------------------- segmented passes

// Geometry of one output tile of a pair given by its item record (the same
// derivation as piece_irregular's).
__device__ __forceinline__ Piece piece_of_item(const SegItem& d, int Tm) {
  Piece p;
  p.src = d.src;
  p.na_tot = d.na;
  p.nb_tot = d.nb;
  p.out0 = d.out0;
  const uint64_t end = d.src + d.na + d.nb;
  const uint64_t start = d.src > d.out0 ? d.src : d.out0;
  const uint64_t stop = end < d.out0 + Tm ? end : d.out0 + Tm;
  p.front = static_cast<uint32_t>(start - d.out0);
  p.d0 = start - d.src;
  p.d1 = stop - d.src;
  p.last = stop == end;
  return p;
}

// Work items of the launch: the merge tiles of the first count_ge[q] listed
// segments.
__device__ __forceinline__ uint64_t seg_pass_items(const SegPassList& L, uint32_t& count) {
  count = __ldg(L.count_ge + L.q);
  return count ? __ldg(L.piece_end + (count - 1)) : 0;
}

// A listed segment in this launch: its range (offsets clamped as the
// segmented sort's plan clamps them), its first tile index, this launch's
// pass j of it, and its first work item and item count.
struct SegPassGeo {
  uint64_t lo, hi, G0, first, items;
  uint32_t j;
};
__device__ __forceinline__ SegPassGeo seg_pass_geo(const SegPassList& L, uint32_t idx) {
  SegPassGeo g;
  const uint32_t s = __ldg(L.order + idx);
  uint64_t lo = __ldg(L.off + s), hi = __ldg(L.off + s + 1);
  lo = lo < L.n ? lo : L.n;
  hi = hi < L.n ? hi : L.n;
  hi = hi > lo ? hi : lo;
  g.lo = lo;
  g.hi = hi;
  g.first = idx ? __ldg(L.piece_end + (idx - 1)) : 0;
  g.items = __ldg(L.piece_end + idx) - g.first;
  const uint64_t T = L.T;
  g.G0 = lo / T;
  const uint64_t tiles = (hi - 1) / T - g.G0 + 1;
  uint32_t P = 0;
  while ((1ull << P) < tiles) ++P;
  g.j = P - L.q + 1;  // listed for this launch: P >= q
  return g;
}

// The pair of runs and the output tile of the segment's merge tile t: pass j
// merges runs of 2^(j-1) tiles of T keys, pairs start at multiples of 2^j
// tiles (clipped to the segment), and a Tm-tile (Tm divides T) lies in one
// pair.
__device__ __forceinline__ SegItem seg_item_at(const SegPassGeo& g, uint64_t t, uint64_t T,
                                               uint64_t Tm) {
  const uint64_t out0 = (g.lo / Tm + t) * Tm;
  const uint64_t pos = out0 > g.lo ? out0 : g.lo;
  const uint64_t r = pos / T - g.G0;  // the segment's tile that holds pos
  const uint64_t t0 = g.G0 + ((r >> g.j) << g.j);
  const uint64_t a0 = t0 * T, a1 = (t0 + (1ull << (g.j - 1))) * T, b1 = (t0 + (1ull << g.j)) * T;
  SegItem d;
  d.src = a0 > g.lo ? a0 : g.lo;
  const uint64_t A1 = a1 < g.hi ? a1 : g.hi;
  const uint64_t B1 = b1 < g.hi ? b1 : g.hi;
  d.na = A1 - d.src;
  d.nb = B1 > A1 ? B1 - A1 : 0;
  d.out0 = out0;
  return d;
}

// The list position of work item 32 c for every chunk c of 32 items (one
// thread per chunk, binary search on the prefix sums), and the merge
// launches' counters cleared.
__global__ void __launch_bounds__(256) seg_chunk_kernel(const SegPassList L) {
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid < kSegMaxPasses + 2) L.next[tid] = 0;
  const uint32_t count = __ldg(L.count_ge + 1);  // every listed segment
  const uint64_t nitems = count ? __ldg(L.piece_end + (count - 1)) : 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t c = tid; c * 32 < nitems; c += stride) {
    uint32_t lo = 0, hi = count - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(L.piece_end + mid) > c * 32) hi = mid; else lo = mid + 1;
    }
    L.chunk_seg[c] = lo;
  }
}

// One thread per work item: its list position from the chunk table and a
// search among the next 32 positions (a listed segment has at least two
// items), the item's pair record, and its exact split (from the source
// buffer's samples when the launch has them, else a full merge-path search).
template <typename K>
__global__ void __launch_bounds__(256) seg_partition_kernel(const MergeArgs a, int Tm,
                                                            const SegPassList L) {
  uint32_t count;
  const uint64_t nitems = seg_pass_items(L, count);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t item = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
       item < nitems; item += stride) {
    uint32_t lo = __ldg(L.chunk_seg + item / 32);
    uint32_t hi = lo + 31 < count - 1 ? lo + 31 : count - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(L.piece_end + mid) > item) hi = mid; else lo = mid + 1;
    }
    const SegPassGeo g = seg_pass_geo(L, lo);
    const SegItem d = seg_item_at(g, item - g.first, L.T, static_cast<uint64_t>(Tm));
    L.items[item] = d;
    const Piece p = piece_of_item(d, Tm);
    const K* A = static_cast<const K*>(a.kin) + p.src;
    const uint64_t slo = p.d0 > p.nb_tot ? p.d0 - p.nb_tot : 0;
    const uint64_t shi = p.d0 < p.na_tot ? p.d0 : p.na_tot;
    uint64_t i;
    if (!a.samples_in ||
        !split_from_run_samples<K, false>(static_cast<const K*>(a.kin),
                                          static_cast<const K*>(a.samples_in), p, p.d0, slo,
                                          shi, 0, i))
      i = merge_path_bs<K, false>(A, A + p.na_tot, p.d0, slo, shi, 0);
    a.splits[item] = i;
  }
}

// CTAs per SM of the persistent loop below: the one-shot merge_kernel's
// residency for the same configuration (its register count as compiled: 32
// for 32-bit keys at E = 16, 48 at E = 32 or for 64-bit keys, 72-80 for 64-bit
// keys with payloads), except 32-bit keys with payloads at 128 threads: 64
// registers and 8 CTAs instead of the one-shot kernel's 56 and 9, which
// spilled in the loop (100,000 segments with payloads: 39.6 against 41.9 ms
// of merge launches).  Left to the compiler the loop took 80-168 registers.
template <typename K, bool PAIRS, int E, int NT>
constexpr int seg_merge_min_ctas() {
  constexpr int regs = sizeof(K) == 4 ? (PAIRS ? 64 : (E == 16 ? 32 : 48))
                                      : (PAIRS ? (NT == 128 ? 72 : 80) : (NT == 128 ? 48 : 64));
  return 65536 / (regs * NT);
}

// Persistent form of merge_kernel over the launch's work items: CTA b takes
// item b first, then untaken items from an atomic counter per launch, so the
// items in flight stay a narrow band of the arrays as in a one-shot launch
// (CTA b taking b, b + gridDim.x, ... lets the CTAs drift apart: 0.47 against
// 0.39 ms per pass of 2^28 keys).  Thread 0 works an item ahead: while the
// current item's bulk copies are in flight it reads the next item's record
// and splits into the other half of a two-entry shared buffer, and claims the
// item after that, whose counter value it needs only an item later.  For
// 32-bit keys without payloads thread 0 also derives that item's windows once
// for the whole CTA (the other threads read them instead of each deriving them
// from 64-bit positions: 0.366 against 0.393 ms per pass of 2^28 keys); with
// payloads every thread derives them (the shared form took 81.0 against 79.8
// ms for 100,000 segments with payloads), and so do 64-bit keys (not measured
// in the shared form).  The mbarrier is initialised once and its phase
// alternates per item.
template <typename K, bool PAIRS, int E, int NT, bool MAP, bool SMP>
__global__ void __launch_bounds__(NT, (seg_merge_min_ctas<K, PAIRS, E, NT>()))
    seg_merge_kernel(const MergeArgs a, const SegPassList L) {
  constexpr bool kShared = !PAIRS && sizeof(K) == 4;  // windows derived by thread 0 for the CTA
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_ok;
  __shared__ TileWindows s_win[kShared ? 2 : 1];
  __shared__ SegItem s_item[kShared ? 1 : 2];
  __shared__ uint64_t s_split[2][2];
  __shared__ uint64_t s_idx[2];
  __shared__ uint64_t s_claim;  // thread 0: the item after the one in the other slot
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
  uint32_t count;
  const uint64_t nitems = seg_pass_items(L, count);
  if (blockIdx.x >= nitems) return;
  const auto fetch = [&](uint32_t slot, uint64_t item) {
    s_idx[slot] = item;
    if (item < nitems) {
      const SegItem d = L.items[item];
      const uint64_t i0 = a.splits[item];
      const uint64_t i1 = item + 1 < nitems ? a.splits[item + 1] : 0;
      if constexpr (kShared) {
        const Piece p = piece_of_item(d, E * NT);
        s_win[slot] = tile_windows<K>(p, i0, p.last ? p.na_tot : i1);
      } else {
        s_item[slot] = d;
        s_split[slot][0] = i0;
        s_split[slot][1] = i1;
      }
    }
  };
  // the record loads and the claim are independent, so their latencies overlap
  // (and both overlap the bulk copies); the claim is kept in shared memory,
  // not in a register live across the merge network
  const auto ahead = [&](uint32_t slot) {
    const uint64_t item = s_claim;
    const uint64_t next = gridDim.x + atomicAdd(L.next + L.q, 1ull);
    fetch(slot, item);
    s_claim = next;
  };
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    s_claim = blockIdx.x;
    ahead(0);
  }
  __syncthreads();
#pragma unroll 1
  for (uint32_t phase = 0; s_idx[phase] < nitems; phase ^= 1u) {
    bool ok;
    if constexpr (kShared) {
      ok = merge_windows<K, PAIRS, E, NT, MAP, SMP ? 2 : 0>(a, s_win[phase], bar, phase,
                                                            smraw + 16, &s_ok,
                                                            [&] { ahead(phase ^ 1u); });
    } else {
      const Piece p = piece_of_item(s_item[phase], E * NT);
      const uint64_t i0 = s_split[phase][0];
      const uint64_t i1 = p.last ? p.na_tot : s_split[phase][1];
      ok = merge_tile<K, PAIRS, E, NT, MAP, SMP ? 2 : 0>(a, p, i0, i1, bar, phase, smraw + 16,
                                                         &s_ok, [&] { ahead(phase ^ 1u); });
    }
    if (!ok) return;
    __syncthreads();  // shared memory is free before the next item's copies land
  }
}

// ---------------------------------------------------------------- segmented-pass launchers

// Grid of the persistent passes: every CTA resident at once.
template <typename F>
static cudaError_t resident_grid(F kern, int threads, size_t smem, unsigned& grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) !=
      cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  grid = static_cast<unsigned>(sms * per_sm);
  return cudaSuccess;
}

cudaError_t launch_seg_chunks(const SegPassList& L, cudaStream_t s) {
  unsigned grid = 0;
  cudaError_t e = resident_grid(seg_chunk_kernel, 256, 0, grid);
  if (e != cudaSuccess) return e;
  seg_chunk_kernel<<<grid, 256, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_seg_partition(int key_bytes, int cfg, const MergeArgs& a,
                                 const SegPassList& L, cudaStream_t s) {
  if (cfg < 0 || cfg >= kNumMergeCfgs) return cudaErrorInvalidValue;
  const int Tm = kMergeCfgs[cfg].tile();
  unsigned grid = 0;
  cudaError_t e;
  if (key_bytes == 4) {
    if ((e = resident_grid(seg_partition_kernel<uint32_t>, 256, 0, grid)) != cudaSuccess) return e;
    seg_partition_kernel<uint32_t><<<grid, 256, 0, s>>>(a, Tm, L);
  } else if (key_bytes == 8) {
    if ((e = resident_grid(seg_partition_kernel<uint64_t>, 256, 0, grid)) != cudaSuccess) return e;
    seg_partition_kernel<uint64_t><<<grid, 256, 0, s>>>(a, Tm, L);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename K, bool PAIRS, int E, int NT, bool MAP, bool SMP>
static cudaError_t launch_sm3(const MergeArgs& a, const SegPassList& L, cudaStream_t s) {
  using S = MergeSmem<K, PAIRS, E, NT>;
  auto kern = seg_merge_kernel<K, PAIRS, E, NT, MAP, SMP>;
  const uint32_t smem = S::kTotal > smem_floor_bytes() ? S::kTotal : smem_floor_bytes();
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  unsigned grid = 0;
  if ((err = resident_grid(kern, NT, smem, grid)) != cudaSuccess) return err;
  MergeArgs b = a;
  b.wait_ns = wait_limit_ns();
  kern<<<grid, NT, smem, s>>>(b, L);
  return cudaGetLastError();
}

template <typename K, bool PAIRS, int E, int NT, bool MAP>
static cudaError_t launch_sm2(const MergeArgs& a, const SegPassList& L, cudaStream_t s) {
  return a.samples_out ? launch_sm3<K, PAIRS, E, NT, MAP, true>(a, L, s)
                       : launch_sm3<K, PAIRS, E, NT, MAP, false>(a, L, s);
}

template <typename K, bool PAIRS, int E, int NT>
static cudaError_t launch_sm(const MergeArgs& a, const SegPassList& L, cudaStream_t s) {
  return (a.mode_in | a.mode_out) != 0 ? launch_sm2<K, PAIRS, E, NT, true>(a, L, s)
                                       : launch_sm2<K, PAIRS, E, NT, false>(a, L, s);
}

template <typename K, bool PAIRS>
static cudaError_t dispatch_sm(int cfg, const MergeArgs& a, const SegPassList& L,
                               cudaStream_t s) {
  switch (cfg) {
    case 0: return launch_sm<K, PAIRS, 16, 256>(a, L, s);
    case 1:
      if constexpr (!PAIRS && sizeof(K) == 4) return launch_sm<K, PAIRS, 32, 128>(a, L, s);
      break;
    case 2:
      if constexpr (!PAIRS && sizeof(K) == 4) return launch_sm<K, PAIRS, 32, 256>(a, L, s);
      break;
    case 3: return launch_sm<K, PAIRS, 16, 128>(a, L, s);
    default: break;
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_seg_merge(int key_bytes, bool pairs, int cfg, const MergeArgs& a,
                             const SegPassList& L, cudaStream_t s) {
  if (!merge_cfg_supported(key_bytes, pairs, cfg)) return cudaErrorInvalidValue;
  if (key_bytes == 4)
    return pairs ? dispatch_sm<uint32_t, true>(cfg, a, L, s)
                 : dispatch_sm<uint32_t, false>(cfg, a, L, s);
  return pairs ? dispatch_sm<uint64_t, true>(cfg, a, L, s)
               : dispatch_sm<uint64_t, false>(cfg, a, L, s);
}

}  // namespace bcf
