// bcf_merge.cu -- BCFMergesort's global merge passes (Sec. 3.2; Lemma 2):
// adjacent sorted runs A, B are merged into one run of |A| + |B| keys with
// coalesced global access and a conflict-free merge in shared memory.
//
// The paper merges each pair with one warp, page by page (Algorithm 6), and
// rebalances the last rounds with a sample-splitter distribution (Algorithm
// 7, Lemma 1).  Here every output tile of Tm keys is an independent CTA: the
// merge-path partition finds, for the tile's first output position d, the
// exact number i of A-keys among the first d outputs -- an exact splitter,
// so every CTA does the same amount of work in every pass, which is what the
// paper's distribution step is for.  The CTA then
//   1. stages its A-window and B-window into shared memory with bulk copies
//      (cp.async.bulk, completion on an mbarrier; 16-byte-misaligned edges
//      are read with plain loads);
//   2. reads the bitonic sequence [pads_min, A, pads_max, reversed B] into
//      registers in STR layout (a warp reads 32 consecutive shared words;
//      rows that contain both A- and B-lanes issue two predicated loads so
//      the two arrays never share a request -- no bank conflicts);
//   3. runs the bitonic merge (log2 Tm stages: register stages, one padded
//      transpose, shuffle stages) -- data-oblivious, so its shared-memory
//      accesses are conflict-free like the paper's ShearSort merge;
//   4. writes its Tm outputs with 128-bit stores.
// Stability: each element carries its rank in the stable merged order (A
// before B on equal keys); the network compares (key, rank).
#include <cuda_runtime.h>

#include <type_traits>

#include "bcf_device.cuh"
#include "bcf_internal.h"

namespace bcf {

// Geometry of one work item: the part of one pair's output that falls into
// one Tm-aligned output tile.
struct Piece {
  uint64_t src;     // index of A[0] in the source array (B[0] = src + na_tot)
  uint64_t na_tot, nb_tot;
  uint64_t out0;    // first index of the Tm-aligned output tile
  uint64_t d0, d1;  // diagonal range of the pair's merged output covered
  uint32_t front;   // tile slots before the piece (filled with -inf pads)
  bool last;        // piece ends at the pair's end
};

__device__ __forceinline__ Piece piece_regular(const MergeArgs& a, uint64_t item, int Tm) {
  Piece p;
  const uint64_t L = a.run;
  const uint64_t out0 = item * static_cast<uint64_t>(Tm);
  const uint64_t pair = out0 / (2 * L);
  p.src = pair * 2 * L;
  const uint64_t left = a.n - p.src;
  p.na_tot = left < L ? left : L;
  const uint64_t rest = left - p.na_tot;
  p.nb_tot = rest < L ? rest : L;
  p.out0 = out0;
  p.front = 0;
  p.d0 = out0 - p.src;
  const uint64_t tot = p.na_tot + p.nb_tot;
  p.d1 = p.d0 + Tm < tot ? p.d0 + Tm : tot;
  p.last = p.d1 == tot;
  return p;
}

__device__ __forceinline__ Piece piece_irregular(const PairList& pl, uint64_t item, int Tm) {
  // last pair whose first piece is <= item
  uint32_t lo = 0, hi = pl.npairs - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (pl.p[mid].piece0 <= item) lo = mid; else hi = mid - 1;
  }
  const PairDesc& d = pl.p[lo];
  Piece p;
  p.src = d.off;
  p.na_tot = d.na;
  p.nb_tot = d.nb;
  const uint64_t end = d.off + d.na + d.nb;
  const uint64_t g = d.off / Tm + (item - d.piece0);
  p.out0 = g * Tm;
  const uint64_t start = d.off > p.out0 ? d.off : p.out0;
  const uint64_t stop = end < p.out0 + Tm ? end : p.out0 + Tm;
  p.front = static_cast<uint32_t>(start - p.out0);
  p.d0 = start - d.off;
  p.d1 = stop - d.off;
  p.last = stop == end;
  return p;
}

// Merge path: number of A-keys among the first d outputs of the stable merge
// (A first on equal keys), i.e. the smallest i with A[i] > B[d-1-i].
template <typename K>
__device__ __forceinline__ uint64_t merge_path(const K* A, uint64_t na, const K* B, uint64_t nb,
                                               uint64_t d, int mode) {
  uint64_t lo = d > nb ? d - nb : 0;
  uint64_t hi = d < na ? d : na;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (map_key(A[mid], mode) > map_key(B[d - 1 - mid], mode))
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

// Regular launches (one sort pass) carry no pair list.
struct NoPairs {
  uint32_t unused;
};
template <bool IRREG>
using PairParam = typename std::conditional<IRREG, PairList, NoPairs>::type;

template <bool IRREG>
__device__ __forceinline__ Piece piece_of(const MergeArgs& a, const PairParam<IRREG>& pl,
                                          uint64_t item, int Tm) {
  if constexpr (IRREG)
    return piece_irregular(pl, item, Tm);
  else
    return piece_regular(a, item, Tm);
}
template <bool IRREG>
__device__ __forceinline__ uint64_t first_item(const PairParam<IRREG>& pl) {
  if constexpr (IRREG)
    return pl.p[0].piece0;
  else
    return 0;
}

template <typename K, bool IRREG>
__global__ void __launch_bounds__(256) partition_kernel(const MergeArgs a, int Tm,
                                                        const __grid_constant__ PairParam<IRREG> pl) {
  const uint64_t local = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (local >= a.nitems) return;
  const uint64_t item = first_item<IRREG>(pl) + local;
  const Piece p = piece_of<IRREG>(a, pl, item, Tm);
  const K* A = static_cast<const K*>(a.kin) + p.src;
  a.splits[item] = merge_path(A, p.na_tot, A + p.na_tot, p.nb_tot, p.d0, a.mode_in);
}

// Stage elements [g0, g1) of `src` (absolute indices; src 16-byte aligned)
// into shared memory at `dst` (16-byte aligned) so that element x lands at
// dst[x - align_down(g0)].  The 16-byte-aligned body goes by bulk copy issued
// by the calling thread; returns its byte count (0 if none).  The ragged tail
// is left to stage_tail().
template <typename T>
__device__ __forceinline__ uint32_t stage_bulk(T* dst, const T* src, uint64_t g0, uint64_t g1,
                                               uint64_t* bar) {
  constexpr uint64_t V = 16 / sizeof(T);
  const uint64_t a0 = g0 & ~(V - 1), a1 = g1 & ~(V - 1);
  if (g1 <= g0 || a1 <= a0) return 0;
  const uint32_t bytes = static_cast<uint32_t>((a1 - a0) * sizeof(T));
  bulk_g2s(dst, src + a0, bytes, bar);
  return bytes;
}
template <typename T>
__device__ __forceinline__ void stage_tail(T* dst, const T* src, uint64_t g0, uint64_t g1,
                                           uint32_t lane) {
  constexpr uint64_t V = 16 / sizeof(T);
  if (g1 <= g0) return;
  const uint64_t a0 = g0 & ~(V - 1), a1 = g1 & ~(V - 1);
  const uint64_t t0 = a1 > g0 ? a1 : g0;
  const uint64_t x = t0 + lane;
  if (lane < V && x < g1) dst[x - a0] = src[x];
}

template <typename K, bool PAIRS, int E, int NT>
struct MergeSmem {
  static constexpr int Tm = E * NT;
  static constexpr int VK = 16 / sizeof(K);
  // staged keys: A and B windows back to back, each 16-byte aligned
  static constexpr uint32_t kKeyBytes = ((Tm + 3 * VK) * sizeof(K) + 15) / 16 * 16;
  static constexpr uint32_t kValBytes = PAIRS ? ((Tm + 12) * 4 + 15) / 16 * 16 : 0;
  static constexpr uint32_t kStageBytes = kKeyBytes + kValBytes;
  static constexpr uint32_t kPlane = padded_words(Tm);
  static constexpr uint32_t kPlaneBytes = Frag<K, PAIRS, E>::W * kPlane * 4;
  static constexpr uint32_t kBody = kStageBytes > kPlaneBytes ? kStageBytes : kPlaneBytes;
  static constexpr uint32_t kTotal = 16 + kBody;  // + mbarrier
};

template <typename K, bool PAIRS, int E, int NT, bool IRREG>
__global__ void __launch_bounds__(NT) merge_kernel(const MergeArgs a,
                                                   const __grid_constant__ PairParam<IRREG> pl) {
  using S = MergeSmem<K, PAIRS, E, NT>;
  constexpr int Tm = S::Tm;
  constexpr uint64_t VK = S::VK;
  extern __shared__ __align__(16) unsigned char smraw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
  unsigned char* body = smraw + 16;
  const uint32_t tid = threadIdx.x;

  const uint64_t item = first_item<IRREG>(pl) + blockIdx.x;
  const Piece p = piece_of<IRREG>(a, pl, item, Tm);
  const uint64_t i0 = a.splits[item];
  const uint64_t i1 = p.last ? p.na_tot : a.splits[item + 1];
  const uint64_t j0 = p.d0 - i0, j1 = p.d1 - i1;
  const uint32_t na = static_cast<uint32_t>(i1 - i0), nb = static_cast<uint32_t>(j1 - j0);
  const uint32_t front = p.front;

  // absolute source index ranges of the two windows
  const uint64_t ga0 = p.src + i0, ga1 = p.src + i1;
  const uint64_t gb0 = p.src + p.na_tot + j0, gb1 = p.src + p.na_tot + j1;
  const uint32_t offA = static_cast<uint32_t>(ga0 & (VK - 1));
  const uint32_t lenA = static_cast<uint32_t>((offA + na + VK - 1) & ~(VK - 1));  // 16B multiple
  const uint32_t offB = static_cast<uint32_t>(gb0 & (VK - 1));
  K* smA = reinterpret_cast<K*>(body);
  K* smB = smA + lenA;
  uint32_t* svA = reinterpret_cast<uint32_t*>(body + S::kKeyBytes);
  const uint32_t offvA = static_cast<uint32_t>(ga0 & 3), offvB = static_cast<uint32_t>(gb0 & 3);
  uint32_t* svB = svA + ((offvA + na + 3) & ~3u);

  const K* kin = static_cast<const K*>(a.kin);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    // the bulk copies' total byte count must be announced before any of them
    // can complete, so sum first, then arm, then issue
    constexpr uint64_t VV = 4;
    auto body_bytes = [](uint64_t g0, uint64_t g1, uint64_t V, uint64_t sz) -> uint32_t {
      const uint64_t a0 = g0 & ~(V - 1), a1 = g1 & ~(V - 1);
      return (g1 > g0 && a1 > a0) ? static_cast<uint32_t>((a1 - a0) * sz) : 0u;
    };
    uint32_t total = body_bytes(ga0, ga1, VK, sizeof(K)) + body_bytes(gb0, gb1, VK, sizeof(K));
    if constexpr (PAIRS)
      total += body_bytes(ga0, ga1, VV, 4) + body_bytes(gb0, gb1, VV, 4);
    mbar_arrive_expect_tx(bar, total);
    stage_bulk(smA, kin, ga0, ga1, bar);
    stage_bulk(smB, kin, gb0, gb1, bar);
    if constexpr (PAIRS) {
      stage_bulk(svA, a.vin, ga0, ga1, bar);
      stage_bulk(svB, a.vin, gb0, gb1, bar);
    }
  } else if (tid >= 32 && tid < 64) {
    const uint32_t lane = tid - 32;
    // lanes 0-7: A keys, 8-15: B keys, 16-23: A values, 24-31: B values
    if (lane < 8) stage_tail(smA, kin, ga0, ga1, lane);
    else if (lane < 16) stage_tail(smB, kin, gb0, gb1, lane - 8);
    else if (PAIRS && lane < 24) stage_tail(svA, a.vin, ga0, ga1, lane - 16);
    else if (PAIRS) stage_tail(svB, a.vin, gb0, gb1, lane - 24);
  }
  if (!mbar_wait_bounded(bar, 0, a.err, kErrTmaTimeout)) {
    // give the copies one more bounded chance to land before the CTA exits
    mbar_wait_bounded(bar, 0, nullptr, 0);
    return;
  }
  __syncthreads();  // tails written with plain stores

  // Read the bitonic sequence into STR registers: k = e*NT + tid.
  //   [0, front)            -inf pads          (rank k)
  //   [front, front+na)     A[k - front]       (rank k)
  //   [front+na, Tm-nb)     +inf pads          (rank Tm + k)
  //   [Tm-nb, Tm)           B[Tm-1-k]          (rank front + na + (Tm-1-k))
  Frag<K, PAIRS, E> f;
  const uint32_t endA = front + na, begB = Tm - nb;
  const uint32_t warp0 = tid & ~31u;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t k = e * NT + tid;
    const uint32_t row0 = e * NT + warp0;
    const bool isA = k >= front && k < endA;
    const bool isB = k >= begB;
    const K pad = k < front ? KeyLimits<K>::kMin : KeyLimits<K>::kMax;
    const K* pa = smA + offA + (k - front);
    const K* pb = smB + offB + (Tm - 1 - k);
    K key;
    if (row0 < endA && row0 + 31 >= begB) {
      key = lds_pred(pa, isA, pad);
      key = lds_pred(pb, isB, key);
    } else {
      key = isA ? *pa : (isB ? *pb : pad);
    }
    f.k[e] = (isA || isB) ? map_key(key, a.mode_in) : key;
    if constexpr (PAIRS) {
      const uint32_t* qa = svA + offvA + (k - front);
      const uint32_t* qb = svB + offvB + (Tm - 1 - k);
      uint32_t val;
      if (row0 < endA && row0 + 31 >= begB) {
        val = lds_pred(qa, isA, 0u);
        val = lds_pred(qb, isB, val);
      } else {
        val = isA ? *qa : (isB ? *qb : 0u);
      }
      f.v[e] = val;
      f.ix[e] = isB ? endA + (Tm - 1 - k) : (k < endA ? k : Tm + k);
    }
  }

  uint32_t* planes = reinterpret_cast<uint32_t*>(body);
  bitonic_merge_str<NT>(f, planes, S::kPlane);

  // outputs: BLK layout, thread holds tile slots tid*E .. tid*E+E-1
  K* kout = static_cast<K*>(a.kout) + p.out0;
  uint32_t* vout = PAIRS ? a.vout + p.out0 : nullptr;
  const uint32_t s0 = tid * E;
  const uint32_t cnt = static_cast<uint32_t>(p.d1 - p.d0);
  if (s0 >= front && s0 + E <= front + cnt) {
    using KV = typename std::conditional<sizeof(K) == 4, uint4, ulonglong2>::type;
#pragma unroll
    for (int q = 0; q < E / static_cast<int>(VK); ++q) {
      KV kv;
      K* kp = reinterpret_cast<K*>(&kv);
#pragma unroll
      for (int c = 0; c < static_cast<int>(VK); ++c)
        kp[c] = unmap_key(f.k[q * VK + c], a.mode_out);
      *reinterpret_cast<KV*>(kout + s0 + q * VK) = kv;
    }
    if constexpr (PAIRS) {
#pragma unroll
      for (int q = 0; q < E / 4; ++q)
        *reinterpret_cast<uint4*>(vout + s0 + 4 * q) =
            make_uint4(f.v[4 * q], f.v[4 * q + 1], f.v[4 * q + 2], f.v[4 * q + 3]);
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t s = s0 + e;
      if (s >= front && s < front + cnt) {
        kout[s] = unmap_key(f.k[e], a.mode_out);
        if constexpr (PAIRS) vout[s] = f.v[e];
      }
    }
  }
}

// ---------------------------------------------------------------- dispatch

bool merge_cfg_supported(int key_bytes, bool pairs, int cfg) {
  if (cfg < 0 || cfg >= kNumMergeCfgs) return false;
  if (key_bytes != 4 && key_bytes != 8) return false;
  return !(pairs && kMergeCfgs[cfg].E > 16);
}

template <typename K, bool PAIRS, int E, int NT>
static cudaError_t launch_m(const MergeArgs& a, const PairList* pl, cudaStream_t s) {
  using S = MergeSmem<K, PAIRS, E, NT>;
  if (a.nitems == 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>(a.nitems);
  cudaError_t err;
  if (pl) {
    auto kern = merge_kernel<K, PAIRS, E, NT, true>;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kTotal);
    if (err != cudaSuccess) return err;
    kern<<<grid, NT, S::kTotal, s>>>(a, *pl);
  } else {
    auto kern = merge_kernel<K, PAIRS, E, NT, false>;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kTotal);
    if (err != cudaSuccess) return err;
    kern<<<grid, NT, S::kTotal, s>>>(a, NoPairs{0});
  }
  return cudaGetLastError();
}

template <typename K, bool PAIRS>
static cudaError_t dispatch_m(int cfg, const MergeArgs& a, const PairList* pl, cudaStream_t s) {
  switch (cfg) {
    case 0: return launch_m<K, PAIRS, 16, 256>(a, pl, s);
    case 1: return launch_m<K, PAIRS, 16, 512>(a, pl, s);
    case 2:
      if constexpr (!PAIRS) return launch_m<K, PAIRS, 32, 256>(a, pl, s);
      break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_merge(int key_bytes, bool pairs, int cfg, const MergeArgs& a,
                         const PairList* pl, cudaStream_t s) {
  if (!merge_cfg_supported(key_bytes, pairs, cfg)) return cudaErrorInvalidValue;
  if (key_bytes == 4)
    return pairs ? dispatch_m<uint32_t, true>(cfg, a, pl, s)
                 : dispatch_m<uint32_t, false>(cfg, a, pl, s);
  return pairs ? dispatch_m<uint64_t, true>(cfg, a, pl, s)
               : dispatch_m<uint64_t, false>(cfg, a, pl, s);
}

cudaError_t launch_partition(int key_bytes, int cfg, const MergeArgs& a, const PairList* pl,
                             cudaStream_t s) {
  if (cfg < 0 || cfg >= kNumMergeCfgs) return cudaErrorInvalidValue;
  if (a.nitems == 0) return cudaSuccess;
  const int Tm = kMergeCfgs[cfg].tile();
  const unsigned grid = static_cast<unsigned>((a.nitems + 255) / 256);
  if (key_bytes == 4) {
    if (pl) partition_kernel<uint32_t, true><<<grid, 256, 0, s>>>(a, Tm, *pl);
    else partition_kernel<uint32_t, false><<<grid, 256, 0, s>>>(a, Tm, NoPairs{0});
  } else {
    if (pl) partition_kernel<uint64_t, true><<<grid, 256, 0, s>>>(a, Tm, *pl);
    else partition_kernel<uint64_t, false><<<grid, 256, 0, s>>>(a, Tm, NoPairs{0});
  }
  return cudaGetLastError();
}

}  // namespace bcf
