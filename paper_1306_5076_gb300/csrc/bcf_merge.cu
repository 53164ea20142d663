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
//   1. stages the keys of its A-window and B-window into shared memory with
//      bulk copies (cp.async.bulk, completion on an mbarrier), each rounded
//      out to whole 16-byte blocks (only the array's last partial block is
//      read with plain loads);
//   2. reads the bitonic sequence [pads_min, A, pads_max, reversed B] into
//      registers in STR layout (a warp reads 32 consecutive shared words;
//      rows that contain both A- and B-lanes issue two predicated loads so
//      the two arrays never share a request -- no bank conflicts);
//   3. runs the bitonic merge: log2 Tm ascending register stages in the STR,
//      MID and BLK layouts joined by two padded, conflict-free transposes --
//      data-oblivious like the paper's ShearSort merge;
//   4. writes its Tm output keys with 32-byte stores, and with payloads reads
//      each output's payload from global memory by its rank and writes those
//      the same way.
// Stability: each element carries its rank in the stable merged order (A
// before B on equal keys); the network compares (key, rank).  The rank also
// names the element's source position, so the payloads need not travel
// through the network.  The tile code lives in bcf_merge.cuh (shared with the
// segmented sort's merge launches).
#include <cuda_runtime.h>

#include <type_traits>

#include "bcf_merge.cuh"

namespace bcf {

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

template <typename K, bool IRREG, bool MAP>
__global__ void __launch_bounds__(256) partition_kernel(const MergeArgs a, int Tm,
                                                        const __grid_constant__ PairParam<IRREG> pl) {
  pdl_wait();
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
    uint64_t i;
    if (a.samples_in && split_from_run_samples<K, MAP>(static_cast<const K*>(a.kin),
                                                       static_cast<const K*>(a.samples_in), p,
                                                       d, lo, hi, a.mode_in, i)) {
      a.splits[item] = i;
      return;
    }
  }
  a.splits[item] = merge_path_bs<K, MAP>(A, B, d, lo, hi, a.mode_in);
}

// SMP (irregular passes): the launch writes samples of its output (a pass
// with a successor); without it the kernel carries no sample code at all.
// Regular passes check for a sample array at run time, as the measured
// sort's passes always have.  One CTA per output tile.
template <typename K, bool PAIRS, int E, int NT, bool IRREG, bool MAP, bool SMP>
__global__ void __launch_bounds__(NT) merge_kernel(const MergeArgs a,
                                                   const __grid_constant__ PairParam<IRREG> pl) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_ok;
  pdl_wait();
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
  const uint64_t item = first_item<IRREG>(pl) + blockIdx.x;
  const Piece p = piece_of<IRREG>(a, pl, item, E * NT);
  const uint64_t i0 = a.splits[item];
  const uint64_t i1 = p.last ? p.na_tot : a.splits[item + 1];
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  merge_tile<K, PAIRS, E, NT, MAP, IRREG ? (SMP ? 2 : 0) : 1>(a, p, i0, i1, bar, 0u, smraw + 16,
                                                              &s_ok, [] {});
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
  return launch_chained(kern, dim3(static_cast<unsigned>(a.nitems)), dim3(NT), smem, s, b, pl);
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
static cudaError_t launch_p(const MergeArgs& a, int Tm, const PairParam<IRREG>& pl,
                            cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>((a.nitems + 255) / 256);
  return launch_chained(partition_kernel<K, IRREG, MAP>, dim3(grid), dim3(256), 0, s, a, Tm, pl);
}

cudaError_t launch_partition(int key_bytes, int cfg, const MergeArgs& a, const PairList* pl,
                             cudaStream_t s) {
  if (cfg < 0 || cfg >= kNumMergeCfgs) return cudaErrorInvalidValue;
  if (a.nitems == 0) return cudaSuccess;
  const int Tm = kMergeCfgs[cfg].tile();
  const bool map = a.mode_in != 0;
  if (key_bytes == 4) {
    if (pl) return map ? launch_p<uint32_t, true, true>(a, Tm, *pl, s)
                       : launch_p<uint32_t, true, false>(a, Tm, *pl, s);
    return map ? launch_p<uint32_t, false, true>(a, Tm, NoPairs{0}, s)
               : launch_p<uint32_t, false, false>(a, Tm, NoPairs{0}, s);
  }
  if (pl) return map ? launch_p<uint64_t, true, true>(a, Tm, *pl, s)
                     : launch_p<uint64_t, true, false>(a, Tm, *pl, s);
  return map ? launch_p<uint64_t, false, true>(a, Tm, NoPairs{0}, s)
             : launch_p<uint64_t, false, false>(a, Tm, NoPairs{0}, s);
}


}  // namespace bcf
