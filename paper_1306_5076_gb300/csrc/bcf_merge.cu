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
//      (cp.async.bulk, completion on an mbarrier), each rounded out to whole
//      16-byte blocks (only the array's last partial block is read with plain
//      loads);
//   2. reads the bitonic sequence [pads_min, A, pads_max, reversed B] into
//      registers in STR layout (a warp reads 32 consecutive shared words;
//      rows that contain both A- and B-lanes issue two predicated loads so
//      the two arrays never share a request -- no bank conflicts);
//   3. runs the bitonic merge: log2 Tm ascending register stages in the STR,
//      MID and BLK layouts joined by two padded, conflict-free transposes --
//      data-oblivious like the paper's ShearSort merge;
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
  // runs are powers of two long: the pair's start is out0 rounded down to 2L
  p.src = (out0 >> (a.run_log2 + 1)) << (a.run_log2 + 1);
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

// Merge path (exact splitter): the number of A-keys among the first d outputs
// of the stable merge (A first on equal keys), i.e. the smallest i with
// A[i] > B[d-1-i], or min(d, |A|) if there is none.  One thread per work item,
// binary search in global memory.  (A warp-cooperative 32-ary search needs
// ~6 instead of ~27 dependent rounds but reads ~7x more sectors, and was
// measured slower at every run length.)
template <typename K, bool MAP>
__device__ __forceinline__ uint64_t merge_path_bs(const K* A, const K* B, uint64_t d, uint64_t lo,
                                                  uint64_t hi, int mode) {
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;  // lo <= mid < hi: A[mid] and B[d-1-mid] exist
    K x = __ldg(A + mid), y = __ldg(B + (d - 1 - mid));
    if constexpr (MAP) {
      x = map_key(x, mode);
      y = map_key(y, mode);
    }
    if (x > y)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

template <typename K, bool IRREG, bool MAP>
__global__ void __launch_bounds__(256) partition_kernel(const MergeArgs a, int Tm,
                                                        const __grid_constant__ PairParam<IRREG> pl) {
  const uint64_t local = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (local >= a.nitems) return;
  const uint64_t item = first_item<IRREG>(pl) + local;
  const Piece p = piece_of<IRREG>(a, pl, item, Tm);
  const K* A = static_cast<const K*>(a.kin) + p.src;
  const K* B = A + p.na_tot;
  const uint64_t d = p.d0;
  const uint64_t lo = d > p.nb_tot ? d - p.nb_tot : 0;
  const uint64_t hi = d < p.na_tot ? d : p.na_tot;
  if constexpr (!IRREG && !MAP) {
    if (a.samples_in) {
      // Merge path of the runs' samples (every S-th key; runs and d are
      // multiples of S), then the exact search only within +-S of it: the
      // true split is within S of S times the samples' split.  The result is
      // checked against the split's defining inequalities; should that fail,
      // the full search below runs.
      constexpr uint64_t S = kSampleStride;
      const K* As = static_cast<const K*>(a.samples_in) + p.src / S;
      const K* Bs = As + p.na_tot / S;
      const uint64_t nas = (p.na_tot + S - 1) / S, nbs = (p.nb_tot + S - 1) / S, D = d / S;
      const uint64_t sa = merge_path_bs<K, false>(As, Bs, D, D > nbs ? D - nbs : 0,
                                                  D < nas ? D : nas, 0);
      const uint64_t wlo = sa * S > lo + S ? sa * S - S : lo;
      const uint64_t whi = sa * S + S < hi ? sa * S + S : hi;
      const uint64_t i = merge_path_bs<K, false>(A, B, d, wlo < whi ? wlo : whi, whi, 0);
      const bool left_ok = i == 0 || d - i >= p.nb_tot || !(__ldg(A + i - 1) > __ldg(B + (d - i)));
      const bool right_ok = i >= p.na_tot || d == i || __ldg(A + i) > __ldg(B + (d - i - 1));
      if (left_ok && right_ok && i >= lo && i <= hi) {
        a.splits[item] = i;
        return;
      }
    }
  } else if constexpr (IRREG) {
    if (a.samples_in) {
      // Runs at any offsets: the samples are the keys at the array positions
      // that are multiples of S, so A's are A[cA + kS] and B's B[cB + kS]
      // with cA, cB < S.  Merge path on them at diagonal
      // D = floor((d - cA - cB) / S) + 1 puts the true split within S of
      // cA + S * (A-samples taken) (checked exhaustively on small runs by the
      // host model of this search); the result is then checked against the
      // split's defining inequalities, with the full search as the fallback.
      constexpr uint64_t S = kRunSampleStride;
      const uint64_t offA = p.src, offB = p.src + p.na_tot;
      const uint64_t gA = (offA + S - 1) / S, gB = (offB + S - 1) / S;
      const uint64_t cA = gA * S - offA, cB = gB * S - offB;
      const uint64_t nas = p.na_tot > cA ? (p.na_tot - cA + S - 1) / S : 0;
      const uint64_t nbs = p.nb_tot > cB ? (p.nb_tot - cB + S - 1) / S : 0;
      const K* As = static_cast<const K*>(a.samples_in) + gA;
      const K* Bs = static_cast<const K*>(a.samples_in) + gB;
      uint64_t D = d >= cA + cB ? (d - cA - cB) / S + 1 : 0;
      D = D < nas + nbs ? D : nas + nbs;
      const uint64_t sa = merge_path_bs<K, false>(As, Bs, D, D > nbs ? D - nbs : 0,
                                                  D < nas ? D : nas, 0);
      const uint64_t c = cA + sa * S;
      const uint64_t wlo0 = c > lo + S ? c - S : lo;
      const uint64_t whi = c + S < hi ? c + S : hi;
      const uint64_t wlo = wlo0 < whi ? wlo0 : whi;
      const int m = MAP ? a.mode_in : 0;
      const uint64_t i = merge_path_bs<K, MAP>(A, B, d, wlo, whi, m);
      const auto key = [m](const K* q) { return MAP ? map_key(__ldg(q), m) : __ldg(q); };
      const bool left_ok = i == 0 || d - i >= p.nb_tot || !(key(A + i - 1) > key(B + (d - i)));
      const bool right_ok = i >= p.na_tot || d == i || key(A + i) > key(B + (d - i - 1));
      if (left_ok && right_ok && i >= lo && i <= hi) {
        a.splits[item] = i;
        return;
      }
    }
  }
  a.splits[item] = merge_path_bs<K, MAP>(A, B, d, lo, hi, a.mode_in);
}

// Stage elements [g0, g1) of `src` (absolute indices into an array of n
// elements; src 16-byte aligned) into shared memory at `dst` (16-byte
// aligned) so that element x lands at dst[x - align_down(g0)].  The bulk copy
// covers the window rounded out to whole 16-byte blocks: the up to V - 1
// elements it reads before g0 and after g1 belong to the same array (the
// neighbouring window) and are never used.  Only where rounding up would pass
// the array's end is the ragged tail left out of the copy and staged by
// stage_tail() -- in the last window of the array alone -- so the CTA's own
// shared stores never overlap its bulk copies anywhere else.
template <typename T>
__device__ __forceinline__ uint64_t bulk_end(uint64_t g1, uint64_t n) {
  constexpr uint64_t V = 16 / sizeof(T);
  const uint64_t up = (g1 + V - 1) & ~(V - 1);
  return up <= n ? up : (g1 & ~(V - 1));
}
template <typename T>
__device__ __forceinline__ uint32_t body_bytes(uint64_t g0, uint64_t g1, uint64_t n) {
  constexpr uint64_t V = 16 / sizeof(T);
  const uint64_t a0 = g0 & ~(V - 1), a1 = bulk_end<T>(g1, n);
  return (g1 > g0 && a1 > a0) ? static_cast<uint32_t>((a1 - a0) * sizeof(T)) : 0u;
}
template <typename T>
__device__ __forceinline__ void stage_bulk(T* dst, const T* src, uint64_t g0, uint64_t g1,
                                           uint64_t n, uint64_t* bar) {
  constexpr uint64_t V = 16 / sizeof(T);
  const uint32_t bytes = body_bytes<T>(g0, g1, n);
  if (bytes) bulk_g2s(dst, src + (g0 & ~(V - 1)), bytes, bar);
}
// The ragged tail of a window that ends in the array's last partial 16-byte
// block: lanes [lane0, lane0 + V) of the calling warp copy its at most V - 1
// elements.  Each window's tail is written by its own shared store
// instruction (a predicated store that only those lanes issue), so the tails
// of two windows never share a request.
template <typename T>
__device__ __forceinline__ void stage_tail(T* dst, const T* src, uint64_t g0, uint64_t g1,
                                           uint64_t n, uint32_t lane, uint32_t lane0) {
  constexpr uint64_t V = 16 / sizeof(T);
  const uint64_t a0 = g0 & ~(V - 1), a1 = bulk_end<T>(g1, n);
  const uint64_t t0 = a1 > g0 ? a1 : g0;
  const uint64_t x = t0 + (lane - lane0);
  const bool mine = g1 > g0 && lane >= lane0 && lane < lane0 + V && x < g1;
  if (!__any_sync(0xFFFFFFFFu, mine)) return;  // no tail here (every window but the last)
  T v = 0;
  if (mine) v = src[x];
  sts_pred(dst + (mine ? x - a0 : 0), mine, v);
}

template <typename K, bool PAIRS, int E, int NT>
struct MergeSmem {
  static constexpr int Tm = E * NT;
  static constexpr int VK = 16 / sizeof(K);
  // staged keys: A and B windows back to back, each 16-byte aligned
  static constexpr uint32_t kKeyBytes = ((Tm + 3 * VK) * sizeof(K) + 15) / 16 * 16;
  static constexpr uint32_t kValBytes = PAIRS ? ((Tm + 12) * 4 + 15) / 16 * 16 : 0;
  static constexpr uint32_t kStageBytes = kKeyBytes + kValBytes;
  static constexpr uint32_t kPlaneBytes = Frag<K, PAIRS, E>::W * Geo<E, NT>::kPlane * 4;
  // the transposes reuse the staging area once it has been read
  static constexpr uint32_t kBody = kStageBytes > kPlaneBytes ? kStageBytes : kPlaneBytes;
  static constexpr uint32_t kTotal = 16 + kBody;  // + mbarrier
};

// Element k of the bitonic sequence [-inf pads | A | +inf pads | reversed B]
// read from the staged windows for a whole warp row (uniform fast paths) or
// lane by lane at the boundaries.
template <typename T>
__device__ __forceinline__ T read_seq(const T* sa, const T* sb, uint32_t k, uint32_t row0,
                                      uint32_t front, uint32_t endA, uint32_t begB,
                                      uint32_t Tm1, T pad_lo, T pad_hi, bool& real) {
  if (row0 >= front && row0 + 32 <= endA) {  // the warp's 32 lanes all read A
    real = true;
    return sa[k - front];
  }
  if (row0 >= begB) {  // all read B, reversed
    real = true;
    return sb[Tm1 - k];
  }
  const bool isA = k >= front && k < endA, isB = k >= begB;
  real = isA || isB;
  T v = lds_pred(sa + (k - front), isA, k < front ? pad_lo : pad_hi);
  return lds_pred(sb + (Tm1 - k), isB, v);
}

// SMP (irregular passes): the launch writes samples of its output (a pass
// with a successor); without it the kernel carries no sample code at all.
// Regular passes check for a sample array at run time, as the measured
// sort's passes always have.
template <typename K, bool PAIRS, int E, int NT, bool IRREG, bool MAP, bool SMP>
__global__ void __launch_bounds__(NT) merge_kernel(const MergeArgs a,
                                                   const __grid_constant__ PairParam<IRREG> pl) {
  using S = MergeSmem<K, PAIRS, E, NT>;
  constexpr int Tm = S::Tm;
  constexpr uint64_t VK = S::VK;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_ok;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
  unsigned char* body = smraw + 16;
  const uint32_t tid = threadIdx.x;

  const uint64_t item = first_item<IRREG>(pl) + blockIdx.x;
  const Piece p = piece_of<IRREG>(a, pl, item, Tm);
  const uint64_t i0 = a.splits[item];
  // For sorted runs the splits grow with the diagonal and nothing below
  // changes i1.  Runs that are not sorted (a broken precondition of
  // bcf_merge_runs) can make neighbouring searches disagree; clamping i1 into
  // the windows i0 allows keeps every staged window inside its run and within
  // the tile's shared memory, so such input gives an undefined order but
  // never an out-of-bounds access.
  uint64_t i1 = p.last ? p.na_tot : a.splits[item + 1];
  {
    const uint64_t lo1 = p.d1 > p.nb_tot && p.d1 - p.nb_tot > i0 ? p.d1 - p.nb_tot : i0;
    const uint64_t hi1 = i0 + (p.d1 - p.d0) < p.na_tot ? i0 + (p.d1 - p.d0) : p.na_tot;
    i1 = i1 < lo1 ? lo1 : (i1 > hi1 ? hi1 : i1);
  }
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
    // the total byte count is announced before any copy can complete
    const uint64_t n = a.n;
    uint32_t total = body_bytes<K>(ga0, ga1, n) + body_bytes<K>(gb0, gb1, n);
    if constexpr (PAIRS)
      total += body_bytes<uint32_t>(ga0, ga1, n) + body_bytes<uint32_t>(gb0, gb1, n);
    mbar_arrive_expect_tx(bar, total);
    stage_bulk(smA, kin, ga0, ga1, n, bar);
    stage_bulk(smB, kin, gb0, gb1, n, bar);
    if constexpr (PAIRS) {
      stage_bulk(svA, a.vin, ga0, ga1, n, bar);
      stage_bulk(svB, a.vin, gb0, gb1, n, bar);
    }
    // one thread waits (bounded); the barrier below releases the others
    bool ok = mbar_wait_bounded(bar, 0, a.err, kErrTmaTimeout, a.wait_ns);
    if (!ok) mbar_wait_bounded(bar, 0, nullptr, 0, a.wait_ns);  // let copies in flight land
    s_ok = ok ? 1 : 0;
  } else if (tid >= 32 && tid < 64) {
    const uint32_t lane = tid - 32;
    // lanes 0-7: A keys, 8-15: B keys, 16-23: A values, 24-31: B values, one
    // store instruction per window
    stage_tail(smA, kin, ga0, ga1, a.n, lane, 0);
    stage_tail(smB, kin, gb0, gb1, a.n, lane, 8);
    if constexpr (PAIRS) {
      stage_tail(svA, a.vin, ga0, ga1, a.n, lane, 16);
      stage_tail(svB, a.vin, gb0, gb1, a.n, lane, 24);
    }
  }
  __syncthreads();
  if (!s_ok) return;

  // Read the bitonic sequence into STR registers: k = e*NT + tid.
  //   [0, front)            -inf pads          (rank k)
  //   [front, front+na)     A[k - front]       (rank k)
  //   [front+na, Tm-nb)     +inf pads          (rank Tm + k)
  //   [Tm-nb, Tm)           B[Tm-1-k]          (rank front + na + (Tm-1-k))
  Frag<K, PAIRS, E> f;
  const uint32_t endA = front + na, begB = Tm - nb;
  const uint32_t warp0 = tid & ~31u;
  const K* sa = smA + offA;
  const K* sb = smB + offB;
  const int mode_in = MAP ? a.mode_in : 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t k = e * NT + tid;
    const uint32_t row0 = e * NT + warp0;
    bool real;
    K key = read_seq<K>(sa, sb, k, row0, front, endA, begB, Tm - 1, KeyLimits<K>::kMin,
                        KeyLimits<K>::kMax, real);
    if constexpr (MAP) key = real ? map_key(key, mode_in) : key;
    f.k[e] = key;
    if constexpr (PAIRS) {
      bool rv;
      f.v[e] = read_seq<uint32_t>(svA + offvA, svB + offvB, k, row0, front, endA, begB, Tm - 1,
                                  0u, 0u, rv);
      f.ix[e] = k >= begB ? endA + (Tm - 1 - k) : (k < endA ? k : Tm + k);
    }
  }

  f.one = g_unit_multiplier;
  bitonic_merge_str<NT, CeForms<K, PAIRS>::kMergeBlk, CeForms<K, PAIRS>::kMergeOth>(
      f, reinterpret_cast<uint32_t*>(body));
  // samples of the output for the next pass's merge-path search: the keys at
  // array positions that are multiples of S, still in mapped order (a pass
  // with a successor writes no unmapped keys)
  if constexpr (!IRREG) {
    if (a.samples_out && ((p.out0 + tid * E) % kSampleStride) == 0 && tid * E < p.d1 - p.d0)
      static_cast<K*>(a.samples_out)[(p.out0 + tid * E) / kSampleStride] = f.k[0];
  } else if constexpr (SMP) {
    if (((p.out0 + tid * E) % kRunSampleStride) == 0 && tid * E >= front &&
        tid * E < front + (p.d1 - p.d0))
      static_cast<K*>(a.samples_out)[(p.out0 + tid * E) / kRunSampleStride] = f.k[0];
  }

  // outputs: BLK layout, thread holds tile slots tid*E .. tid*E+E-1
  K* kout = static_cast<K*>(a.kout) + p.out0;
  uint32_t* vout = PAIRS ? a.vout + p.out0 : nullptr;
  const uint32_t s0 = tid * E;
  const uint32_t cnt = static_cast<uint32_t>(p.d1 - p.d0);
  const int mode_out = MAP ? a.mode_out : 0;
  if (s0 >= front && s0 + E <= front + cnt) {
    // out0 and s0 are multiples of 32 bytes: the base pointers decide alignment
    if constexpr (MAP) {
#pragma unroll
      for (int e = 0; e < E; ++e) f.k[e] = unmap_key(f.k[e], mode_out);  // last use of f.k
    }
    store_run<E>(kout + s0, f.k, is_aligned32(a.kout));
    if constexpr (PAIRS) store_run<E>(vout + s0, f.v, is_aligned32(a.vout));
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t s = s0 + e;
      if (s >= front && s < front + cnt) {
        kout[s] = MAP ? unmap_key(f.k[e], mode_out) : f.k[e];
        if constexpr (PAIRS) vout[s] = f.v[e];
      }
    }
  }
}

// Samples of the keys of a merge's given runs (its first pass; later passes
// get theirs from the merge kernel).
template <typename K, bool MAP>
__global__ void __launch_bounds__(256) sample_span_kernel(const K* keys, K* samples, int mode,
                                                          uint64_t g0, uint64_t count) {
  const uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const uint64_t g = g0 + t;
  const K k = keys[g * kRunSampleStride];
  samples[g] = MAP ? map_key(k, mode) : k;
}

template <typename K>
static cudaError_t launch_ss(const void* keys, void* samples, int mode, uint64_t lo, uint64_t hi,
                             cudaStream_t s) {
  constexpr uint64_t S = kRunSampleStride;
  const uint64_t g0 = (lo + S - 1) / S, g1 = (hi + S - 1) / S;
  if (g1 <= g0) return cudaSuccess;
  const uint64_t count = g1 - g0;
  const unsigned grid = static_cast<unsigned>((count + 255) / 256);
  if (mode)
    sample_span_kernel<K, true><<<grid, 256, 0, s>>>(static_cast<const K*>(keys),
                                                     static_cast<K*>(samples), mode, g0, count);
  else
    sample_span_kernel<K, false><<<grid, 256, 0, s>>>(static_cast<const K*>(keys),
                                                      static_cast<K*>(samples), mode, g0, count);
  return cudaGetLastError();
}

cudaError_t launch_sample_span(int key_bytes, const void* keys, void* samples, int mode,
                               uint64_t lo, uint64_t hi, cudaStream_t s) {
  if (key_bytes == 4) return launch_ss<uint32_t>(keys, samples, mode, lo, hi, s);
  if (key_bytes == 8) return launch_ss<uint64_t>(keys, samples, mode, lo, hi, s);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- dispatch

// Pairs and 64-bit keys are built with E = 16 only (register budget).
bool merge_cfg_supported(int key_bytes, bool pairs, int cfg) {
  if (cfg < 0 || cfg >= kNumMergeCfgs) return false;
  if (key_bytes != 4 && key_bytes != 8) return false;
  if (pairs || key_bytes == 8) return kMergeCfgs[cfg].E == 16;
  return true;
}

template <typename K, bool PAIRS, int E, int NT, bool IRREG, bool MAP, bool SMP>
static cudaError_t launch_m3(const MergeArgs& a, const PairParam<IRREG>& pl, cudaStream_t s) {
  using S = MergeSmem<K, PAIRS, E, NT>;
  auto kern = merge_kernel<K, PAIRS, E, NT, IRREG, MAP, SMP>;
  const uint32_t smem = S::kTotal > smem_floor_bytes() ? S::kTotal : smem_floor_bytes();
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  MergeArgs b = a;
  b.wait_ns = wait_limit_ns();
  kern<<<static_cast<unsigned>(a.nitems), NT, smem, s>>>(b, pl);
  return cudaGetLastError();
}

template <typename K, bool PAIRS, int E, int NT, bool IRREG, bool MAP>
static cudaError_t launch_m2(const MergeArgs& a, const PairParam<IRREG>& pl, cudaStream_t s) {
  if (IRREG && !a.samples_out) return launch_m3<K, PAIRS, E, NT, IRREG, MAP, false>(a, pl, s);
  return launch_m3<K, PAIRS, E, NT, IRREG, MAP, true>(a, pl, s);
}

template <typename K, bool PAIRS, int E, int NT>
static cudaError_t launch_m(const MergeArgs& a, const PairList* pl, cudaStream_t s) {
  if (a.nitems == 0) return cudaSuccess;
  const bool map = (a.mode_in | a.mode_out) != 0;
  if (pl)
    return map ? launch_m2<K, PAIRS, E, NT, true, true>(a, *pl, s)
               : launch_m2<K, PAIRS, E, NT, true, false>(a, *pl, s);
  return map ? launch_m2<K, PAIRS, E, NT, false, true>(a, NoPairs{0}, s)
             : launch_m2<K, PAIRS, E, NT, false, false>(a, NoPairs{0}, s);
}

template <typename K, bool PAIRS>
static cudaError_t dispatch_m(int cfg, const MergeArgs& a, const PairList* pl, cudaStream_t s) {
  switch (cfg) {
    case 0: return launch_m<K, PAIRS, 16, 256>(a, pl, s);
    case 1:
      if constexpr (!PAIRS && sizeof(K) == 4) return launch_m<K, PAIRS, 32, 128>(a, pl, s);
      break;
    case 2:
      if constexpr (!PAIRS && sizeof(K) == 4) return launch_m<K, PAIRS, 32, 256>(a, pl, s);
      break;
    case 3: return launch_m<K, PAIRS, 16, 128>(a, pl, s);
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

template <typename K, bool IRREG, bool MAP>
static void launch_p(const MergeArgs& a, int Tm, const PairParam<IRREG>& pl, cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>((a.nitems + 255) / 256);
  partition_kernel<K, IRREG, MAP><<<grid, 256, 0, s>>>(a, Tm, pl);
}

cudaError_t launch_partition(int key_bytes, int cfg, const MergeArgs& a, const PairList* pl,
                             cudaStream_t s) {
  if (cfg < 0 || cfg >= kNumMergeCfgs) return cudaErrorInvalidValue;
  if (a.nitems == 0) return cudaSuccess;
  const int Tm = kMergeCfgs[cfg].tile();
  const bool map = a.mode_in != 0;
  if (key_bytes == 4) {
    if (pl) map ? launch_p<uint32_t, true, true>(a, Tm, *pl, s)
                : launch_p<uint32_t, true, false>(a, Tm, *pl, s);
    else map ? launch_p<uint32_t, false, true>(a, Tm, NoPairs{0}, s)
             : launch_p<uint32_t, false, false>(a, Tm, NoPairs{0}, s);
  } else {
    if (pl) map ? launch_p<uint64_t, true, true>(a, Tm, *pl, s)
                : launch_p<uint64_t, true, false>(a, Tm, *pl, s);
    else map ? launch_p<uint64_t, false, true>(a, Tm, NoPairs{0}, s)
             : launch_p<uint64_t, false, false>(a, Tm, NoPairs{0}, s);
  }
  return cudaGetLastError();
}

}  // namespace bcf
