// bcf_segmented.cuh -- device code of the segmented sort (see bcf_segmented.cu).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "bcf_device.cuh"
#include "bcf_internal.h"

namespace bcf {

constexpr uint32_t kTinyMax = 512;      // keys per tiny segment (32 lanes x 16)
// tiny segments per work item: one per warp of the worker CTA (NT / 32)
constexpr uint32_t kErrQueueTimeout = 2u;
constexpr uint32_t kErrQueueOverflow = 4u;

enum : uint32_t { kWTiny = 1, kWTile = 2, kWPiece = 3, kReady = 0x80000000u };

struct SegWork {
  uint32_t meta;  // kReady | pass << 8 | type
  uint32_t seg;
  uint64_t arg;   // tile / output-tile index relative to the segment, or tiny group
};

struct SegCtl {
  unsigned long long head;     // next slot to take
  unsigned long long reserve;  // slots published or being published
  unsigned long long total;    // work items that will ever exist
  unsigned long long n_tiny;
  unsigned long long tiles;    // tile sorts: queue slots [0, tiles)
};

__host__ __device__ constexpr uint32_t ceil_log2(uint64_t x) {
  uint32_t p = 0;
  while ((1ull << p) < x) ++p;
  return p;
}

struct SegGeo {
  uint64_t lo, hi;
  uint32_t tiles, passes, pieces;
  bool tiny;
};

// skip_odd: segments with an odd index are left as they are (treated as
// empty); used by the pivot-bucket sort, whose odd buckets hold keys equal to
// a splitter and are final after the distribution.
__device__ __forceinline__ SegGeo seg_geo(const uint64_t* off, uint64_t s, uint64_t n, uint32_t T,
                                          bool skip_odd) {
  SegGeo g;
  uint64_t lo = __ldcg(off + s), hi = __ldcg(off + s + 1);
  // memory safety for malformed offsets: clamp into [0, n] and make hi >= lo
  lo = lo < n ? lo : n;
  hi = hi < n ? hi : n;
  hi = hi > lo ? hi : lo;
  if (skip_odd && (s & 1u)) hi = lo;
  g.lo = lo;
  g.hi = hi;
  const uint64_t size = hi - lo;
  g.tiny = size > 0 && size <= kTinyMax;
  g.tiles = (size == 0 || g.tiny) ? 0 : static_cast<uint32_t>((hi - 1) / T - lo / T + 1);
  g.passes = g.tiles > 1 ? ceil_log2(g.tiles) : 0;
  g.pieces = g.tiles;  // merge output tiles: the same T-aligned tiles as the sort
  return g;
}

struct SegArgs {
  const void* kin;
  const uint32_t* vin;
  void* kout;
  uint32_t* vout;
  void* kbuf;      // ping-pong copy (workspace)
  uint32_t* vbuf;
  const uint64_t* off;
  uint64_t nseg, n;
  int mode;
  int skip_odd;  // odd-indexed segments are left untouched
  SegWork* queue;
  uint64_t capacity;
  uint32_t* items_left;
  uint32_t* tiny_list;
  uint64_t* tile_base;    // per segment: its first tile's index among all segments' tiles
  uint64_t* piece_split;  // per tile: merge-path split (A-keys before the piece) of its piece
  SegCtl* ctl;
  uint32_t* err;
  uint64_t wait_ns;       // limit of every wait for a queue slot
  // Merge passes outside the worker (Tm != 0): segments of two or more tiles
  // are block-sorted here and listed for launches of the merge kernel.
  uint32_t Tm;            // their merge tile, or 0: the worker merges
  uint32_t* order;        // listed segments, most passes first
  uint64_t* piece_end;    // inclusive prefix sums of their Tm-tiles in list order
  uint32_t* count_ge;     // [q]: listed segments with q or more passes
  void* samples_out;      // listed segments: tile samples of the output buffer ...
  void* samples_buf;      // ... and of the workspace copy (or nullptr: none)
};

// The plan kernel lives in bcf_segmented.cu.
cudaError_t launch_plan(const SegArgs& a, uint32_t T, uint32_t tiny_per_group, cudaStream_t s);

// ---------------------------------------------------------------- tiny segments

// Sort of one tiny segment (<= 512 keys) by one warp: 16 registers per lane,
// Batcher's network per lane, then bitonic merges across lanes with the
// level's flip as a mirrored shuffle, so every compare-exchange ascends.
template <typename K, bool PAIRS, bool MAP>
__device__ __forceinline__ void warp_sort_segment(const SegArgs& a, uint64_t lo, uint64_t hi) {
  constexpr int E = 16;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t size = static_cast<uint32_t>(hi - lo);
  const K* kin = static_cast<const K*>(a.kin) + lo;
  Frag<K, PAIRS, E> f;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t k = e * 32 + lane;
    const bool real = k < size;
    K x = KeyLimits<K>::kMax;
    if (real) x = MAP ? map_key(__ldcg(kin + k), a.mode) : __ldcg(kin + k);
    f.k[e] = x;
    if constexpr (PAIRS) {
      f.v[e] = real ? __ldcg(a.vin + lo + k) : 0u;
      f.ix[e] = k;
    }
  }
  thread_sort(f, false);
#pragma unroll 1
  for (int j = 5; j <= 9; ++j) {
    // flip: my register e meets the mirrored lane's register 15 - e
    {
      const uint32_t m = (1u << (j - 4)) - 1u;
      const bool upper = (lane & (1u << (j - 5))) != 0;
      K pk[E];
      uint32_t pi[PAIRS ? E : 1], pv[PAIRS ? E : 1];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        pk[e] = __shfl_xor_sync(0xFFFFFFFFu, f.k[E - 1 - e], m);
        if constexpr (PAIRS) {
          pi[e] = __shfl_xor_sync(0xFFFFFFFFu, f.ix[E - 1 - e], m);
          pv[e] = __shfl_xor_sync(0xFFFFFFFFu, f.v[E - 1 - e], m);
        }
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {
        if constexpr (!PAIRS) {
          const K x = f.k[e], y = pk[e];
          f.k[e] = upper ? (x > y ? x : y) : (x < y ? x : y);
        } else {
          const bool p_after = after(pk[e], pi[e], f.k[e], f.ix[e]);
          const bool take = upper ? p_after : !p_after;
          f.k[e] = take ? pk[e] : f.k[e];
          f.ix[e] = take ? pi[e] : f.ix[e];
          f.v[e] = take ? pv[e] : f.v[e];
        }
      }
    }
    // half-cleaners on lane bits j-2 .. 4
#pragma unroll 1
    for (int b = j - 2; b >= 4; --b) {
      const uint32_t m = 1u << (b - 4);
      const bool upper = (lane & m) != 0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const K y = __shfl_xor_sync(0xFFFFFFFFu, f.k[e], m);
        if constexpr (!PAIRS) {
          const K x = f.k[e];
          f.k[e] = upper ? (x > y ? x : y) : (x < y ? x : y);
        } else {
          const uint32_t yi = __shfl_xor_sync(0xFFFFFFFFu, f.ix[e], m);
          const uint32_t yv = __shfl_xor_sync(0xFFFFFFFFu, f.v[e], m);
          const bool p_after = after(y, yi, f.k[e], f.ix[e]);
          const bool take = upper ? p_after : !p_after;
          f.k[e] = take ? y : f.k[e];
          f.ix[e] = take ? yi : f.ix[e];
          f.v[e] = take ? yv : f.v[e];
        }
      }
    }
    // register bits 3 .. 0
#pragma unroll
    for (int q = 3; q >= 0; --q) {
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (!(e & (1 << q))) ce(f, e, e | (1 << q), false);
    }
  }
  K* kout = static_cast<K*>(a.kout) + lo;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t k = lane * E + e;
    if (k < size) {
      kout[k] = MAP ? unmap_key(f.k[e], a.mode) : f.k[e];
      if constexpr (PAIRS) a.vout[lo + k] = f.v[e];
    }
  }
}

// Stores a thread's E consecutive tile slots k0 .. k0+E-1 (BLK layout) of
// which [front, front + cnt) are real: 32-byte vector stores when all E are
// real and the buffers are 32-byte aligned (tiles start at multiples of T),
// else one store per real slot.  ks: the keys; vs: the payloads (PAIRS).
template <int E, bool PAIRS, typename K>
__device__ __forceinline__ void store_slots(K* kdst, uint32_t* vdst, const K* ks,
                                            const uint32_t* vs, uint32_t k0, uint32_t front,
                                            uint32_t cnt, const void* kbase,
                                            const uint32_t* vbase) {
  if (k0 >= front && k0 + E <= front + cnt && is_aligned32(kbase) &&
      (!PAIRS || is_aligned32(vbase))) {
    store_run<E>(kdst + k0, ks, true);
    if constexpr (PAIRS) store_run<E>(vdst + k0, vs, true);
    return;
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t k = k0 + e;
    if (k >= front && k < front + cnt) {
      kdst[k] = ks[e];
      if constexpr (PAIRS) vdst[k] = vs[e];
    }
  }
}

// ---------------------------------------------------------------- tile sort

template <typename K, bool PAIRS, int E, int NT, bool MAP>
__device__ __forceinline__ void sort_tile_item(const SegArgs& a, const SegGeo& g, uint64_t q,
                                               uint32_t* sm) {
  constexpr uint32_t T = E * NT;
  constexpr int V = 16 / sizeof(K);  // keys per 16-byte vector
  using KV = typename VecOf<K, V>::T;
  using VV = typename ValVec<V>::T;
  // with payloads the network sorts (key, position) only: the tile's payloads
  // wait in a padded plane behind the network's planes (the space the
  // payload-carrying merge pieces' third plane takes) and each output's
  // payload is read from there by its position once the tile is sorted (the
  // network's barriers order the plane's writes before the reads)
  Frag<K, PAIRS, E, /*VALS=*/false> f;
  uint32_t* sv = sm + Frag<K, PAIRS, E, false>::W * padded_words(T);
  f.one = g_unit_multiplier;
  const uint32_t tid = threadIdx.x;
  const uint64_t base = (g.lo / T + q) * T;
  const uint64_t s0 = g.lo > base ? g.lo : base;
  const uint64_t s1 = g.hi < base + T ? g.hi : base + T;
  const uint32_t front = static_cast<uint32_t>(s0 - base), cnt = static_cast<uint32_t>(s1 - s0);
  const K* kin = static_cast<const K*>(a.kin) + base;
  const uint32_t* vin = PAIRS ? a.vin + base : nullptr;
  // Thread tid loads the V-element vectors at tile positions
  // pos = q * V * NT + V * tid (coalesced 16-byte loads, as the block sort
  // kernel reads); the position is also the element's rank in the stable
  // input order.  A tile clipped by the segment reads element by element:
  // -inf pads before the segment, +inf pads after it.
  if (front == 0 && cnt == T) {  // kin and vin are 16-byte aligned, base a multiple of T
#pragma unroll
    for (int r = 0; r < E / V; ++r) {
      const uint32_t pos = r * V * NT + V * tid;
      const KV kv = __ldcg(reinterpret_cast<const KV*>(kin + pos));
      const K* kp = reinterpret_cast<const K*>(&kv);
#pragma unroll
      for (int c = 0; c < V; ++c) f.k[r * V + c] = MAP ? map_key(kp[c], a.mode) : kp[c];
      if constexpr (PAIRS) {
        const VV vv = __ldcg(reinterpret_cast<const VV*>(vin + pos));
        const uint32_t* vp = reinterpret_cast<const uint32_t*>(&vv);
#pragma unroll
        for (int c = 0; c < V; ++c) {
          f.ix[r * V + c] = pos + c;
          sv[pos + c + ((pos + c) >> 5)] = vp[c];
        }
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t pos = (e / V) * V * NT + V * tid + (e % V);
      const bool real = pos >= front && pos < front + cnt;
      K x = pos < front ? KeyLimits<K>::kMin : KeyLimits<K>::kMax;
      if (real) x = MAP ? map_key(__ldcg(kin + pos), a.mode) : __ldcg(kin + pos);
      f.k[e] = x;
      if constexpr (PAIRS) {
        f.ix[e] = pos;
        sv[pos + (pos >> 5)] = real ? __ldcg(vin + pos) : 0u;
      }
    }
  }
  block_sort_tile<NT, CeForms<K, PAIRS>::kBlockBlk, CeForms<K, PAIRS>::kBlockOth>(f, sm);
  // the segment's passes alternate buffers so that its last one writes the output
  const bool to_out = (g.passes % 2) == 0;
  K* kout = static_cast<K*>(to_out ? a.kout : a.kbuf) + base;
  uint32_t* vout = PAIRS ? (to_out ? a.vout : a.vbuf) + base : nullptr;
  const bool last = g.passes == 0;
  // samples for the first merge pass's partition when the passes run as
  // launches: the key at every array position that is a multiple of
  // kRunSampleStride, in the buffer this tile is written to (mapped keys)
  void* samples = to_out ? a.samples_out : a.samples_buf;
  const uint32_t p0 = tid * E;
  if (samples && !last && ((base + p0) % kRunSampleStride) == 0 && p0 >= front &&
      p0 < front + cnt)
    static_cast<K*>(samples)[(base + p0) / kRunSampleStride] = f.k[0];
  if constexpr (MAP) {
    if (last) {
#pragma unroll
      for (int e = 0; e < E; ++e) f.k[e] = unmap_key(f.k[e], a.mode);  // last use of f.k
    }
  }
  uint32_t vg[PAIRS ? E : 1];
  if constexpr (PAIRS) {
#pragma unroll
    for (int e = 0; e < E; ++e) vg[e] = sv[f.ix[e] + (f.ix[e] >> 5)];
  }
  store_slots<E, PAIRS>(kout, vout, f.k, vg, p0, front, cnt, to_out ? a.kout : a.kbuf,
                        PAIRS ? (to_out ? a.vout : a.vbuf) : nullptr);
}

// ---------------------------------------------------------------- merge piece

// Merge path by one warp, 32-ary (see partition_kernel in bcf_merge.cu for
// the predicate); A and B are read with .cg loads.
template <typename K>
__device__ __forceinline__ uint64_t warp_merge_path(const K* A, uint64_t na, const K* B,
                                                    uint64_t nb, uint64_t d) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t lo = d > nb ? d - nb : 0;
  uint64_t hi = d < na ? d : na;
  while (lo < hi) {
    const uint64_t span = hi - lo;
    const uint64_t pos = lo + (span * lane) / 32;
    const bool p = __ldcg(A + pos) > __ldcg(B + (d - 1 - pos));
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, p);
    if (m == 0) {
      lo = lo + (span * 31) / 32 + 1;
    } else {
      const int fl = __ffs(m) - 1;
      const uint64_t pf = lo + (span * fl) / 32;
      if (fl > 0) lo = lo + (span * (fl - 1)) / 32 + 1;
      hi = pf;
    }
  }
  return lo;
}

// Geometry of merge piece `rel` of pass `pass` of a segment: the pair of
// input runs A = [A0, A0 + na), B = [A0 + na, A0 + na + nb) it draws from and
// the diagonals [d0, d1) of their merged order that land in its T-aligned
// output tile gt.
struct PieceGeo {
  uint64_t gt, A0, na, nb, ps, pe, d0, d1;
};
__device__ __forceinline__ PieceGeo piece_geo(const SegGeo& g, uint32_t pass, uint64_t rel,
                                              uint64_t T) {
  PieceGeo p;
  const uint64_t G0 = g.lo / T;
  p.gt = G0 + rel;                              // absolute output tile
  const uint64_t q = rel >> pass;               // pair index within the segment
  const uint64_t half = 1ull << (pass - 1);     // tiles per input run
  const uint64_t a0 = (G0 + (q << pass)) * T;
  p.A0 = a0 > g.lo ? a0 : g.lo;
  const uint64_t a1 = (G0 + (q << pass) + half) * T;
  const uint64_t A1 = a1 < g.hi ? a1 : g.hi;
  const uint64_t b1 = (G0 + ((q + 1) << pass)) * T;
  const uint64_t B1 = b1 < g.hi ? b1 : g.hi;
  p.na = A1 - p.A0;
  p.nb = B1 > A1 ? B1 - A1 : 0;
  p.ps = p.gt * T > p.A0 ? p.gt * T : p.A0;
  p.pe = (p.gt + 1) * T < p.A0 + p.na + p.nb ? (p.gt + 1) * T : p.A0 + p.na + p.nb;
  p.d0 = p.ps - p.A0;
  p.d1 = p.pe - p.A0;
  return p;
}

// The merge passes alternate between the output and the workspace copy so
// that the last pass writes the output: pass p reads what pass p-1 wrote.
__device__ __forceinline__ bool pass_reads_out(const SegGeo& g, uint32_t pass) {
  return ((g.passes - (pass - 1)) % 2) == 0;
}

// The two splits of one piece of a long segment, searched by warps 0 and 1
// (out of line: the common path, published splits, keeps its registers).
template <typename K>
__device__ __noinline__ void search_piece_splits(const K* A, uint64_t na, uint64_t nb,
                                                 uint64_t d0, uint64_t d1, uint64_t* s_split) {
  const uint32_t w = threadIdx.x >> 5;
  if (w < 2) {
    const uint64_t d = w == 0 ? d0 : d1;
    const uint64_t i = (w == 1 && d1 == na + nb) ? na : warp_merge_path(A, na, A + na, nb, d);
    if ((threadIdx.x & 31u) == 0) s_split[w] = i;
  }
}

// Whether the CTA that publishes a pass of this segment also finds the
// pass's splits: up to 16 rounds of its warps (a few tens of microseconds).
// A longer segment's pieces search their own, in parallel, so that a single
// huge segment is not held up by one CTA.
template <int NT>
__device__ __forceinline__ bool splits_published(const SegGeo& g) {
  return g.pieces <= 16u * (NT / 32);
}

// Run by the whole CTA that completed a segment's pass `pass - 1`, before it
// publishes pass `pass`: the split (A-keys before the piece's first output)
// of every piece of the pass, one warp per piece, stored per tile.  Each piece
// then reads its start split and the next piece's (or |A| at its pair's end)
// instead of searching for them itself.
template <typename K, int NT>
__device__ __forceinline__ void publish_splits(const SegArgs& a, const SegGeo& g, uint64_t seg,
                                               uint32_t pass, uint64_t T) {
  const uint32_t warp = threadIdx.x >> 5;
  const K* src = static_cast<const K*>(pass_reads_out(g, pass) ? a.kout : a.kbuf);
  const uint64_t tb = __ldcg(a.tile_base + seg);
  for (uint64_t rel = warp; rel < g.pieces; rel += NT / 32) {
    const PieceGeo p = piece_geo(g, pass, rel, T);
    const K* A = src + p.A0;
    const uint64_t i0 = warp_merge_path(A, p.na, A + p.na, p.nb, p.d0);
    if ((threadIdx.x & 31u) == 0) a.piece_split[tb + rel] = i0;
  }
  __threadfence();  // every split is visible before the pass is published
}

template <typename K, bool PAIRS, int E, int NT, bool MAP>
__device__ __forceinline__ void merge_piece_item(const SegArgs& a, const SegGeo& g,
                                                 uint64_t seg, uint32_t pass, uint64_t rel,
                                                 uint32_t* sm, uint64_t* s_split) {
  constexpr uint64_t T = E * NT;  // merge tile == sort tile here
  const uint32_t tid = threadIdx.x;
  const PieceGeo pg = piece_geo(g, pass, rel, T);
  const uint64_t gt = pg.gt, A0 = pg.A0, na = pg.na, nb = pg.nb;
  const uint64_t ps = pg.ps, pe = pg.pe, d0 = pg.d0, d1 = pg.d1;
  const uint64_t A1 = A0 + na;
  const bool src_out = pass_reads_out(g, pass);
  const bool dst_out = ((g.passes - pass) % 2) == 0;
  const K* src = static_cast<const K*>(src_out ? a.kout : a.kbuf);
  const uint32_t* vsrc = PAIRS ? (src_out ? a.vout : a.vbuf) : nullptr;
  uint64_t i0, i1;
  if (splits_published<NT>(g)) {
    // splits published with the pass (publish_splits); the next piece of the
    // same pair starts where this one ends
    const uint64_t tb = __ldcg(a.tile_base + seg);
    i0 = __ldcg(a.piece_split + tb + rel);
    i1 = d1 == na + nb ? na : __ldcg(a.piece_split + tb + rel + 1);
  } else {
    // a long segment: two warps search this piece's two splits
    search_piece_splits(src + A0, na, nb, d0, d1, s_split);
    __syncthreads();
    i0 = s_split[0];
    i1 = s_split[1];
  }
  const uint32_t wa = static_cast<uint32_t>(i1 - i0);
  const uint32_t wb = static_cast<uint32_t>((d1 - i1) - (d0 - i0));
  const uint32_t front = static_cast<uint32_t>(ps - gt * T);
  const uint32_t endA = front + wa, begB = static_cast<uint32_t>(T) - wb;
  const uint64_t ja = A0 + i0, jb = A1 + (d0 - i0);  // first A / B window element
  // Per-thread bases, so that slot k = e*NT + tid of the sequence is read at a
  // base plus the compile-time offset e*NT: A[k - front] from pA[e*NT],
  // reversed B[T-1-k] from pB[-e*NT].  (Integer arithmetic: a base may lie
  // outside the arrays; only slots of the windows are dereferenced.)
  const auto at = [](const void* base, uint64_t idx, uint64_t bytes) {
    return reinterpret_cast<uintptr_t>(base) + idx * bytes;
  };
  const uint64_t ia = ja + tid - front, ib = jb + (T - 1) - tid;
  const K* pA = reinterpret_cast<const K*>(at(src, ia, sizeof(K)));
  const K* pB = reinterpret_cast<const K*>(at(src, ib, sizeof(K)));
  const uint32_t* qA = PAIRS ? reinterpret_cast<const uint32_t*>(at(vsrc, ia, 4)) : nullptr;
  const uint32_t* qB = PAIRS ? reinterpret_cast<const uint32_t*>(at(vsrc, ib, 4)) : nullptr;
  const uint32_t rel0 = tid - front;  // k - front at e = 0 (wraps for k < front)
  Frag<K, PAIRS, E> f;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t k = e * NT + tid;
    const bool isA = rel0 + static_cast<uint32_t>(e * NT) < wa;  // front <= k < endA
    const bool isB = k >= begB;
    K x = k < front ? KeyLimits<K>::kMin : KeyLimits<K>::kMax;
    if (isA) x = __ldcg(pA + e * NT);
    else if (isB) x = __ldcg(pB - e * NT);
    f.k[e] = x;
    if constexpr (PAIRS) {
      uint32_t v = 0u;
      if (isA) v = __ldcg(qA + e * NT);
      else if (isB) v = __ldcg(qB - e * NT);
      f.v[e] = v;
      f.ix[e] = isB ? endA + (static_cast<uint32_t>(T) - 1 - k) : (k < endA ? k : T + k);
    }
  }
  f.one = g_unit_multiplier;
  bitonic_merge_str<NT, CeForms<K, PAIRS>::kPieceBlk, CeForms<K, PAIRS>::kPieceOth>(f, sm);
  K* dst = static_cast<K*>(dst_out ? a.kout : a.kbuf) + gt * T;
  uint32_t* vdst = PAIRS ? (dst_out ? a.vout : a.vbuf) + gt * T : nullptr;
  const bool last = pass == g.passes;
  const uint32_t cnt = static_cast<uint32_t>(pe - ps);
  if constexpr (MAP) {
    if (last) {
#pragma unroll
      for (int e = 0; e < E; ++e) f.k[e] = unmap_key(f.k[e], a.mode);  // last use of f.k
    }
  }
  store_slots<E, PAIRS>(dst, vdst, f.k, PAIRS ? f.v : nullptr, tid * E, front, cnt,
                        dst_out ? a.kout : a.kbuf, PAIRS ? (dst_out ? a.vout : a.vbuf) : nullptr);
}

// ---------------------------------------------------------------- worker

__device__ __forceinline__ bool wait_ready(const SegWork* slot, uint32_t* err, uint64_t limit_ns) {
  const volatile uint32_t* meta = &slot->meta;
  if (*meta & kReady) return true;
  const uint64_t t0 = globaltimer_ns();
  while (!(*meta & kReady)) {
    if (globaltimer_ns() - t0 > limit_ns) {
      atomicOr(err, kErrQueueTimeout);
      return false;
    }
    __nanosleep(200);
  }
  return true;
}

// The worker loop; the kernels below differ only in their register budget.
template <typename K, bool PAIRS, int E, int NT, bool MAP>
__device__ __forceinline__ void seg_worker_body(const SegArgs& a) {
  constexpr uint32_t T = E * NT;
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ SegWork s_w;
  __shared__ int s_go;
  __shared__ int s_publish;
  __shared__ unsigned long long s_base;
  __shared__ uint64_t s_split[2];
  const uint32_t tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      const unsigned long long idx = atomicAdd(&a.ctl->head, 1ull);
      int go = 0;
      if (idx < __ldcg(&a.ctl->total) && wait_ready(a.queue + idx, a.err, a.wait_ns)) {
        __threadfence();
        // the slot may have been written by another SM during this launch
        SegWork w;
        w.meta = *const_cast<const volatile uint32_t*>(&a.queue[idx].meta);
        w.seg = __ldcg(&a.queue[idx].seg);
        w.arg = __ldcg(&a.queue[idx].arg);
        s_w = w;
        go = 1;
      }
      s_go = go;
    }
    __syncthreads();
    if (!s_go) return;
    const SegWork w = s_w;
    const uint32_t type = w.meta & 0xFFu, pass = (w.meta >> 8) & 0xFFu;
    if (type == kWTiny) {
      constexpr uint32_t kPerGroup = NT / 32;
      const uint64_t t = w.arg * kPerGroup + (tid >> 5);
      if (t < __ldcg(&a.ctl->n_tiny)) {
        const uint32_t s = __ldcg(a.tiny_list + t);
        const SegGeo g = seg_geo(a.off, s, a.n, T, a.skip_odd != 0);
        warp_sort_segment<K, PAIRS, MAP>(a, g.lo, g.hi);
      }
      __syncthreads();
      continue;
    }
    const SegGeo g = seg_geo(a.off, w.seg, a.n, T, a.skip_odd != 0);
    if (type == kWTile)
      sort_tile_item<K, PAIRS, E, NT, MAP>(a, g, w.arg, sm);
    else
      merge_piece_item<K, PAIRS, E, NT, MAP>(a, g, w.seg, pass, w.arg, sm, s_split);
    __syncthreads();  // every store of this item is issued
    if (tid == 0) {
      __threadfence();  // ... and visible before the completion is counted
      const uint32_t left = atomicSub(a.items_left + w.seg, 1u);
      s_publish = left == 1 && pass < g.passes && a.Tm == 0;
    }
    __syncthreads();
    if (s_publish) {
      // last item of this pass: the CTA finds the next pass's splits, then
      // publishes the segment's next pass
      if (splits_published<NT>(g)) publish_splits<K, NT>(a, g, w.seg, pass + 1, T);
      const uint32_t m = g.pieces;
      if (tid == 0) {
        a.items_left[w.seg] = m;
        s_base = atomicAdd(&a.ctl->reserve, static_cast<unsigned long long>(m));
        if (s_base + m > a.capacity) atomicOr(a.err, kErrQueueOverflow);
      }
      __syncthreads();
      // every thread publishes a share of the pass's slots: each writes its
      // slots' contents, makes them visible, then sets their ready bits (a
      // segment of 2^31 keys publishes 524,288 slots per pass)
      const unsigned long long base = s_base;
      if (base + m <= a.capacity) {
        for (uint32_t j = tid; j < m; j += NT) {
          a.queue[base + j].seg = w.seg;
          a.queue[base + j].arg = j;
        }
        __threadfence();
        for (uint32_t j = tid; j < m; j += NT)
          *const_cast<volatile uint32_t*>(&a.queue[base + j].meta) =
              kReady | ((pass + 1) << 8) | kWPiece;
      }
    }
    __syncthreads();
  }
}

// 32-bit keys without payloads: at least 1152 / NT CTAs per SM (at most 56
// registers a thread for 128 threads, 64 for 256 and 512), so the 128-thread
// configuration runs 9 or more CTAs per SM and the 256-thread one 4.  Left to
// the compiler they took 128 registers and half the CTAs, and the sort of
// 100,000 segments ran 52 ms instead of 37 ms.  Payloads and 64-bit keys need
// more registers than that.
template <typename K, bool PAIRS, int E, int NT, bool MAP>
__global__ void __launch_bounds__(NT, 1152 / NT) seg_worker_capped(const SegArgs a) {
  seg_worker_body<K, PAIRS, E, NT, MAP>(a);
}
// Payloads and 64-bit keys: at least 768 / NT CTAs per SM (at most 80
// registers a thread for 256 threads, 3 CTAs per SM, against 122 registers
// and 2 CTAs left to the compiler).  The few spilled words stay in L1:
// 100,000 segments with u32 payloads took 106.5 ms against 124.9 ms (a
// 64-register cap: 106.7 ms).
constexpr int kSegWideThreads = 768;
template <typename K, bool PAIRS, int E, int NT, bool MAP>
__global__ void __launch_bounds__(NT, kSegWideThreads / NT) seg_worker(const SegArgs a) {
  seg_worker_body<K, PAIRS, E, NT, MAP>(a);
}
template <typename K, bool PAIRS, int E, int NT, bool MAP>
constexpr auto seg_kernel() {
  if constexpr (!PAIRS && sizeof(K) == 4)
    return &seg_worker_capped<K, PAIRS, E, NT, MAP>;
  else
    return &seg_worker<K, PAIRS, E, NT, MAP>;
}

// Listed segments (merge passes outside the worker): nothing is published
// during the sort, every tile sort and tiny segment is known from the plan,
// so they run as two plain launches instead of the persistent worker.
// Tile sorts: one CTA per queue slot [0, tiles) -- the block sort kernel's
// shape and register budget (the worker's budget also covers its merge
// pieces and the warp sorts, which halved the CTAs per SM).
template <typename K, bool PAIRS, int E, int NT, bool MAP>
__global__ void __launch_bounds__(NT) seg_tile_kernel(const SegArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  const uint64_t idx = blockIdx.x;
  if (idx >= __ldcg(&a.ctl->tiles)) return;
  const uint32_t seg = __ldcg(&a.queue[idx].seg);
  const uint64_t q = __ldcg(&a.queue[idx].arg);
  const SegGeo g = seg_geo(a.off, seg, a.n, E * NT, a.skip_odd != 0);
  sort_tile_item<K, PAIRS, E, NT, MAP>(a, g, q, sm);
}
// Tiny segments: one warp each, over the plan's list of them.
template <typename K, bool PAIRS, bool MAP>
__global__ void __launch_bounds__(256) seg_tiny_kernel(const SegArgs a, uint32_t T) {
  const uint64_t ntiny = __ldcg(&a.ctl->n_tiny);
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x / 32);
  for (uint64_t t = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / 32;
       t < ntiny; t += warps) {
    const SegGeo g = seg_geo(a.off, __ldcg(a.tiny_list + t), a.n, T, a.skip_odd != 0);
    warp_sort_segment<K, PAIRS, MAP>(a, g.lo, g.hi);
  }
}

template <typename K, bool PAIRS, int E, int NT, bool MAP>
cudaError_t launch_seg(const SegArgs& a, cudaStream_t s) {
  // W planes: the merge pieces' (key, rank, payload) words, or the tile
  // sorts' (key, position) words and their payload plane
  constexpr int W = Frag<K, PAIRS, E>::W;
  static_assert(W >= Frag<K, PAIRS, E, false>::W + (PAIRS ? 1 : 0), "tile sort planes");
  const size_t smem = static_cast<size_t>(W) * Geo<E, NT>::kPlane * sizeof(uint32_t);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t err;
  if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return err;
  if (a.Tm) {
    // listed segments: plan, tile sorts, tiny segments
    auto tk = seg_tile_kernel<K, PAIRS, E, NT, MAP>;
    if ((err = cudaFuncSetAttribute(tk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem))) != cudaSuccess)
      return err;
    if ((err = launch_plan(a, E * NT, NT / 32, s)) != cudaSuccess) return err;
    // a segment touches at most size / T + 2 tiles
    const uint64_t tiles_bound = a.n / (E * NT) + 2 * a.nseg + 2;
    tk<<<static_cast<unsigned>(tiles_bound), NT, smem, s>>>(a);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    auto yk = seg_tiny_kernel<K, PAIRS, MAP>;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, yk, 256, 0)) != cudaSuccess)
      return err;
    yk<<<sms * (per_sm > 0 ? per_sm : 1), 256, 0, s>>>(a, E * NT);
    return cudaGetLastError();
  }
  auto kern = seg_kernel<K, PAIRS, E, NT, MAP>();
  if ((err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem))) != cudaSuccess)
    return err;
  if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) !=
      cudaSuccess)
    return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if ((err = launch_plan(a, E * NT, NT / 32, s)) != cudaSuccess) return err;
  kern<<<sms * per_sm, NT, smem, s>>>(a);  // one co-resident wave
  return cudaGetLastError();
}

template <typename K, bool PAIRS, bool MAP>
cudaError_t dispatch_seg(int cfg, const SegArgs& a, cudaStream_t s) {
  switch (cfg) {
    case 0: return launch_seg<K, PAIRS, 16, 256, MAP>(a, s);
    case 1: return launch_seg<K, PAIRS, 16, 128, MAP>(a, s);
    case 2:
      if constexpr (!PAIRS && sizeof(K) == 4) return launch_seg<K, PAIRS, 32, 128, MAP>(a, s);
      break;
    case 3:  // larger tiles: more bytes per work item's latency chain
      if constexpr (!PAIRS && sizeof(K) == 4) return launch_seg<K, PAIRS, 32, 256, MAP>(a, s);
      break;
    case 4:
      if constexpr (!PAIRS && sizeof(K) == 4) return launch_seg<K, PAIRS, 32, 512, MAP>(a, s);
      break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

// 32-bit keys without payloads in mapped order (f32, i32, descending) are
// instantiated in bcf_segmented_u32m.cu, in parallel with the rest.
extern template cudaError_t dispatch_seg<uint32_t, false, true>(int, const SegArgs&, cudaStream_t);

// Launch of the persistent sort for key type K and payload flag PAIRS
// (instantiated in bcf_segmented_u32.cu, _u32p.cu, _u64.cu and _u64p.cu so
// that the four compile in parallel).
template <typename K, bool PAIRS>
cudaError_t launch_segmented_kp(int cfg, const SegArgs& a, cudaStream_t s) {
  return a.mode != 0 ? dispatch_seg<K, PAIRS, true>(cfg, a, s)
                     : dispatch_seg<K, PAIRS, false>(cfg, a, s);
}

extern template cudaError_t launch_segmented_kp<uint32_t, false>(int, const SegArgs&, cudaStream_t);
extern template cudaError_t launch_segmented_kp<uint32_t, true>(int, const SegArgs&, cudaStream_t);
extern template cudaError_t launch_segmented_kp<uint64_t, false>(int, const SegArgs&, cudaStream_t);
extern template cudaError_t launch_segmented_kp<uint64_t, true>(int, const SegArgs&, cudaStream_t);

}  // namespace bcf
