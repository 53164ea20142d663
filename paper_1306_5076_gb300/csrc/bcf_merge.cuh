// bcf_merge.cuh -- device code shared by the merge passes of a sort or a merge
// of runs (bcf_merge.cu) and the merge passes of a segmented sort's multi-tile
// segments (bcf_seg_merge.cu): a work item's geometry, the merge-path split
// search, the bulk staging of the two windows and the merge of one output
// tile (Sec. 3.2; Lemma 2).
#pragma once
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

// The split at diagonal d of piece p's pair (runs at any offsets), from the
// samples of the source array: the keys at the array positions that are
// multiples of S = kRunSampleStride, so A's are A[cA + kS] and B's
// B[cB + kS] with cA, cB < S.  Merge path on them at diagonal
// D = floor((d - cA - cB) / S) + 1 puts the true split within S of
// cA + S * (A-samples taken) (checked exhaustively on small runs by the host
// model of this search); the search within that window is then checked
// against the split's defining inequalities.  Returns false when the check
// fails (the caller searches in full).
template <typename K, bool MAP>
__device__ __forceinline__ bool split_from_run_samples(const K* kin, const K* samples,
                                                       const Piece& p, uint64_t d, uint64_t lo,
                                                       uint64_t hi, int mode, uint64_t& out) {
  constexpr uint64_t S = kRunSampleStride;
  const K* A = kin + p.src;
  const K* B = A + p.na_tot;
  const uint64_t offA = p.src, offB = p.src + p.na_tot;
  const uint64_t gA = (offA + S - 1) / S, gB = (offB + S - 1) / S;
  const uint64_t cA = gA * S - offA, cB = gB * S - offB;
  const uint64_t nas = p.na_tot > cA ? (p.na_tot - cA + S - 1) / S : 0;
  const uint64_t nbs = p.nb_tot > cB ? (p.nb_tot - cB + S - 1) / S : 0;
  const K* As = samples + gA;
  const K* Bs = samples + gB;
  uint64_t D = d >= cA + cB ? (d - cA - cB) / S + 1 : 0;
  D = D < nas + nbs ? D : nas + nbs;
  const uint64_t sa = merge_path_bs<K, false>(As, Bs, D, D > nbs ? D - nbs : 0,
                                              D < nas ? D : nas, 0);
  const uint64_t c = cA + sa * S;
  const uint64_t wlo0 = c > lo + S ? c - S : lo;
  const uint64_t whi = c + S < hi ? c + S : hi;
  const uint64_t wlo = wlo0 < whi ? wlo0 : whi;
  const int m = MAP ? mode : 0;
  const uint64_t i = merge_path_bs<K, MAP>(A, B, d, wlo, whi, m);
  const auto key = [m](const K* q) { return MAP ? map_key(__ldg(q), m) : __ldg(q); };
  const bool left_ok = i == 0 || d - i >= p.nb_tot || !(key(A + i - 1) > key(B + (d - i)));
  const bool right_ok = i >= p.na_tot || d == i || key(A + i) > key(B + (d - i - 1));
  out = i;
  return left_ok && right_ok && i >= lo && i <= hi;
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

// Shared memory of one merge tile.  Only keys are staged: with payloads the
// network carries (key, rank), and each output's payload is read from global
// memory by its rank once the tile is merged (moving the payload through the
// network took 0.918 against 0.850 ms per pass of 2^28 u32 pairs).
template <typename K, bool PAIRS, int E, int NT>
struct MergeSmem {
  static constexpr int Tm = E * NT;
  static constexpr int VK = 16 / sizeof(K);
  // staged keys: A and B windows back to back, each 16-byte aligned
  static constexpr uint32_t kKeyBytes = ((Tm + 3 * VK) * sizeof(K) + 15) / 16 * 16;
  static constexpr uint32_t kStageBytes = kKeyBytes;
  static constexpr uint32_t kPlaneBytes =
      Frag<K, PAIRS, E, /*VALS=*/false>::W * Geo<E, NT>::kPlane * 4;
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

// The two windows of one output tile -- the piece p of a pair whose A-window
// starts at split i0 and ends at split i1 -- and where their keys are staged
// in the tile's shared memory, with the tile's output start and count.  For
// sorted runs the splits grow with the diagonal and the clamp below changes
// nothing.  Runs that are not sorted (a broken precondition of
// bcf_merge_runs) can make neighbouring searches disagree; clamping i1 into
// the windows i0 allows keeps every staged window inside its run and within
// the tile's shared memory, so such input gives an undefined order but never
// an out-of-bounds access.
struct TileWindows {
  uint64_t ga0, ga1, gb0, gb1;  // absolute source index ranges of the A and B windows
  uint64_t out0;                // first index of the Tm-aligned output tile
  uint32_t na, nb, front, cnt;  // window lengths; real output slots [front, front + cnt)
  uint32_t offA, lenA, offB;    // staged layout: A at offA, B at lenA + offB (elements)
};
template <typename K>
__device__ __forceinline__ TileWindows tile_windows(const Piece& p, uint64_t i0, uint64_t i1) {
  constexpr uint64_t VK = 16 / sizeof(K);
  {
    const uint64_t lo1 = p.d1 > p.nb_tot && p.d1 - p.nb_tot > i0 ? p.d1 - p.nb_tot : i0;
    const uint64_t hi1 = i0 + (p.d1 - p.d0) < p.na_tot ? i0 + (p.d1 - p.d0) : p.na_tot;
    i1 = i1 < lo1 ? lo1 : (i1 > hi1 ? hi1 : i1);
  }
  TileWindows w;
  const uint64_t j0 = p.d0 - i0, j1 = p.d1 - i1;
  w.na = static_cast<uint32_t>(i1 - i0);
  w.nb = static_cast<uint32_t>(j1 - j0);
  w.front = p.front;
  w.cnt = static_cast<uint32_t>(p.d1 - p.d0);
  w.out0 = p.out0;
  w.ga0 = p.src + i0;
  w.ga1 = p.src + i1;
  w.gb0 = p.src + p.na_tot + j0;
  w.gb1 = p.src + p.na_tot + j1;
  w.offA = static_cast<uint32_t>(w.ga0 & (VK - 1));
  w.lenA = static_cast<uint32_t>((w.offA + w.na + VK - 1) & ~(VK - 1));  // 16B multiple
  w.offB = static_cast<uint32_t>(w.gb0 & (VK - 1));
  return w;
}

// Thread 0: announce the tile's byte count on `bar`, then bulk-copy its two
// key windows (A at body, B right after A's 16-byte-rounded span).
template <typename K>
__device__ __forceinline__ void stage_issue(const MergeArgs& a, const TileWindows& w,
                                            unsigned char* body, uint64_t* bar) {
  K* smA = reinterpret_cast<K*>(body);
  const K* kin = static_cast<const K*>(a.kin);
  const uint64_t n = a.n;
  // the total byte count is announced before any copy can complete
  mbar_arrive_expect_tx(bar, body_bytes<K>(w.ga0, w.ga1, n) + body_bytes<K>(w.gb0, w.gb1, n));
  stage_bulk(smA, kin, w.ga0, w.ga1, n, bar);
  stage_bulk(smA + w.lenA, kin, w.gb0, w.gb1, n, bar);
}

// Warp 1 (lane = threadIdx.x - 32): the key windows' ragged tails at the
// array's end.  Lanes 0-7: A, 8-15: B, one store instruction per window.
template <typename K>
__device__ __forceinline__ void stage_tails(const MergeArgs& a, const TileWindows& w,
                                            unsigned char* body, uint32_t lane) {
  K* smA = reinterpret_cast<K*>(body);
  const K* kin = static_cast<const K*>(a.kin);
  stage_tail(smA, kin, w.ga0, w.ga1, a.n, lane, 0);
  stage_tail(smA + w.lenA, kin, w.gb0, w.gb1, a.n, lane, 8);
}

// A tile whose B window (or A window) is empty -- every tile of sorted or
// reversed stretches and of long runs of equal keys -- is the other window
// itself: slot s in [front, front + cnt) is its element s - front.  Its keys
// come from the staged window and its payloads from global memory, both in
// rows of 32 consecutive slots per warp instruction, with no network at all
// (in the network's BLK output order a warp's payload loads would sit E
// words apart, on two L1 banks).  Samples as merge_staged writes them.
template <typename K, bool PAIRS, int E, int NT, bool MAP, int SAMPLES>
__device__ __forceinline__ void copy_staged(const MergeArgs& a, const TileWindows& w,
                                            const unsigned char* body) {
  const uint32_t tid = threadIdx.x;
  const uint32_t front = w.front, cnt = w.cnt;
  const bool from_a = w.nb == 0;
  const K* st = reinterpret_cast<const K*>(body) + (from_a ? w.offA : w.lenA + w.offB) - front;
  const int mode_in = MAP ? a.mode_in : 0, mode_out = MAP ? a.mode_out : 0;
  // samples: the (mapped) key of slot tid * E, as the network's BLK output has it
  if constexpr (SAMPLES != 0) {
    const uint32_t p = tid * E;
    constexpr uint32_t S = SAMPLES == 1 ? kSampleStride : kRunSampleStride;
    const bool want = SAMPLES == 1 ? (a.samples_out != nullptr && p < cnt)
                                   : (p >= front && p < front + cnt);
    if (want && ((w.out0 + p) % S) == 0) {
      const K x = st[p];
      static_cast<K*>(a.samples_out)[(w.out0 + p) / S] = MAP ? map_key(x, mode_in) : x;
    }
  }
  K* kout = static_cast<K*>(a.kout) + w.out0 + tid;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t s = e * NT + tid;
    if (s - front < cnt) {
      const K x = st[s];
      kout[e * NT] = MAP ? unmap_key(map_key(x, mode_in), mode_out) : x;
    }
  }
  if constexpr (PAIRS) {
    const uint32_t* src = a.vin + ((from_a ? w.ga0 : w.gb0) - front) + tid;
    uint32_t* dst = a.vout + w.out0 + tid;
    uint32_t vg[E];
#pragma unroll
    for (int e = 0; e < E; ++e) vg[e] = (e * NT + tid - front < cnt) ? __ldg(src + e * NT) : 0u;
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e * NT + tid - front < cnt) dst[e * NT] = vg[e];
  }
}

// The merge of a staged tile (its key windows landed in `body`, visible to
// every thread): the bitonic sequence of (key, rank) read into registers, the
// network (whose transposes reuse `body`), the samples and the key stores,
// then -- with payloads -- each output's payload read by its rank and stored.
//   sequence slot k = e*NT + tid (STR layout):
//   [0, front)            -inf pads          (rank k)
//   [front, front+na)     A[k - front]       (rank k)
//   [front+na, Tm-nb)     +inf pads          (rank Tm + k)
//   [Tm-nb, Tm)           B[Tm-1-k]          (rank front + na + (Tm-1-k))
// A rank in [front, endA) is then A's element rank - front, a rank in
// [endA, endA + nb) B's element rank - endA; the pads' ranks lie outside both
// and pads never reach a real output slot.  SAMPLES: 0 writes none, 1 writes
// regular-pass samples when a.samples_out is set, 2 writes samples at array
// positions that are multiples of kRunSampleStride (irregular passes with a
// successor).
template <typename K, bool PAIRS, int E, int NT, bool MAP, int SAMPLES>
__device__ __forceinline__ void merge_staged(const MergeArgs& a, const TileWindows& w,
                                             unsigned char* body) {
  constexpr int Tm = E * NT;
  const uint32_t tid = threadIdx.x;
  const uint32_t na = w.na, nb = w.nb, front = w.front, cnt = w.cnt;
  const uint64_t out0 = w.out0;
  Frag<K, PAIRS, E, /*VALS=*/false> f;
  const uint32_t endA = front + na, begB = Tm - nb;
  const uint32_t warp0 = tid & ~31u;
  const K* sa = reinterpret_cast<const K*>(body) + w.offA;
  const K* sb = reinterpret_cast<const K*>(body) + w.lenA + w.offB;
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
    if constexpr (PAIRS) f.ix[e] = k >= begB ? endA + (Tm - 1 - k) : (k < endA ? k : Tm + k);
  }

  f.one = g_unit_multiplier;
  bitonic_merge_str<NT, CeForms<K, PAIRS>::kMergeBlk, CeForms<K, PAIRS>::kMergeOth>(
      f, reinterpret_cast<uint32_t*>(body));
  // samples of the output for the next pass's merge-path search: the keys at
  // array positions that are multiples of S, still in mapped order (a pass
  // with a successor writes no unmapped keys)
  if constexpr (SAMPLES == 1) {
    if (a.samples_out && ((out0 + tid * E) % kSampleStride) == 0 && tid * E < cnt)
      static_cast<K*>(a.samples_out)[(out0 + tid * E) / kSampleStride] = f.k[0];
  } else if constexpr (SAMPLES == 2) {
    if (((out0 + tid * E) % kRunSampleStride) == 0 && tid * E >= front && tid * E < front + cnt)
      static_cast<K*>(a.samples_out)[(out0 + tid * E) / kRunSampleStride] = f.k[0];
  }

  // outputs: BLK layout, thread holds tile slots tid*E .. tid*E+E-1
  K* kout = static_cast<K*>(a.kout) + out0;
  const uint32_t s0 = tid * E;
  const bool full = s0 >= front && s0 + E <= front + cnt;
  const int mode_out = MAP ? a.mode_out : 0;
  if (full) {
    // out0 and s0 are multiples of 32 bytes: the base pointers decide alignment
    if constexpr (MAP) {
#pragma unroll
      for (int e = 0; e < E; ++e) f.k[e] = unmap_key(f.k[e], mode_out);  // last use of f.k
    }
    store_run<E>(kout + s0, f.k, is_aligned32(a.kout));
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t s = s0 + e;
      if (s >= front && s < front + cnt) kout[s] = MAP ? unmap_key(f.k[e], mode_out) : f.k[e];
    }
  }
  if constexpr (PAIRS) {
    // payloads by rank, once the keys are stored (their registers are free)
    uint32_t* vout = a.vout + out0;
    uint32_t vg[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t s = s0 + e, r = f.ix[e];
      const uint64_t src = r < endA ? w.ga0 + (r - front) : w.gb0 + (r - endA);
      vg[e] = (s >= front && s < front + cnt) ? __ldg(a.vin + src) : 0u;
    }
    if (full) {
      store_run<E>(vout + s0, vg, is_aligned32(a.vout));
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const uint32_t s = s0 + e;
        if (s >= front && s < front + cnt) vout[s] = vg[e];
      }
    }
  }
}

// One output tile, staged and merged by the calling CTA: thread 0 stages the
// key windows with bulk copies completing on `bar` (initialised by the
// caller) and waits for phase parity `phase`; warp 1 stages the ragged tails.
// Returns false when the wait for the bulk copies ran out (the error word is
// set; the caller's CTA stops).  Thread 0 calls on_issued() once its bulk
// copies are issued, before it waits for them.  The windows come derived
// (the segmented sort's persistent merge: thread 0 derives them once for the
// CTA) ...
template <typename K, bool PAIRS, int E, int NT, bool MAP, int SAMPLES, typename OnIssued>
__device__ __forceinline__ bool merge_windows(const MergeArgs& a, const TileWindows& w,
                                              uint64_t* bar, uint32_t phase,
                                              unsigned char* body, int* s_ok,
                                              OnIssued&& on_issued) {
  const uint32_t tid = threadIdx.x;
  if (tid == 0) {
    stage_issue<K>(a, w, body, bar);
    on_issued();
    // one thread waits (bounded); the barrier below releases the others
    bool ok = mbar_wait_bounded(bar, phase, a.err, kErrTmaTimeout, a.wait_ns);
    if (!ok) mbar_wait_bounded(bar, phase, nullptr, 0, a.wait_ns);  // let copies in flight land
    *s_ok = ok ? 1 : 0;
  } else if (tid >= 32 && tid < 64) {
    stage_tails<K>(a, w, body, tid - 32);
  }
  __syncthreads();
  if (!*s_ok) return false;
  if (w.na == 0 || w.nb == 0)
    copy_staged<K, PAIRS, E, NT, MAP, SAMPLES>(a, w, body);
  else
    merge_staged<K, PAIRS, E, NT, MAP, SAMPLES>(a, w, body);
  return true;
}

// ... or every thread derives them from the piece p of a pair whose A-window
// starts at split i0 and ends at split i1 (the one-shot kernels, whose pieces
// come from the block index).
template <typename K, bool PAIRS, int E, int NT, bool MAP, int SAMPLES, typename OnIssued>
__device__ __forceinline__ bool merge_tile(const MergeArgs& a, const Piece& p, uint64_t i0,
                                           uint64_t i1, uint64_t* bar, uint32_t phase,
                                           unsigned char* body, int* s_ok, OnIssued&& on_issued) {
  return merge_windows<K, PAIRS, E, NT, MAP, SAMPLES>(a, tile_windows<K>(p, i0, i1), bar, phase,
                                                      body, s_ok, on_issued);
}

}  // namespace bcf
