// bcf_block_sort.cu -- the base case: every tile of T consecutive keys (plus
// payloads) sorted inside one CTA without a single shared-memory bank
// conflict (Sec. 3.1, "Base case"; Algorithms 1, 2 and 5).
//
// The paper sorts a w x w matrix in shared memory with ShearSort: register
// Batcher networks on rows and columns, transposes in between, and shifted
// diagonals so no transpose conflicts.  On sm_103a the same principles are
// kept -- data-oblivious register networks, one thread per row/column of a
// skewed shared-memory matrix -- but ShearSort's O(log w) row/column rounds
// are replaced by a bitonic sort whose cross-thread stages are warp shuffles
// (no shared memory at all) or a single padded transpose, which needs far
// fewer compare-exchanges per key for tiles of 4K-16K keys.
//
//   1. coalesced 128-bit loads straight into registers (each thread takes V
//      consecutive keys from every NT*V-key stripe); keys are mapped to
//      unsigned order (f32 totalOrder, descending);
//   2. Batcher odd-even merge sort of the thread's E registers;
//   3. bitonic merge levels j = r+1 .. t in BLK layout, using the STR layout
//      (one padded transpose each way) for the levels' top bits;
//   4. 128-bit stores of the thread's E consecutive outputs.
// Pairs carry a tie-break index (input position in the tile) so that the
// result is the stable order.
#include <cuda_runtime.h>

#include "bcf_device.cuh"
#include "bcf_internal.h"

namespace bcf {

// Full bitonic sort of the CTA's E*NT elements.  On entry each thread's E
// registers hold arbitrary elements; on exit the tile is ascending in BLK
// layout (thread tid holds sorted positions tid*E .. tid*E + E - 1).
template <int NT, typename K, bool PAIRS, int E>
__device__ __forceinline__ void block_bitonic_sort(Frag<K, PAIRS, E>& f, uint32_t* sm,
                                                   uint32_t plane) {
  constexpr int r = ilog2(E), t = ilog2(E * NT);
  static_assert(t <= 2 * r + 5, "tile too large for two layouts");
  static_assert(E <= 32, "direction masks hold 32 registers");
  const uint32_t tid = threadIdx.x;
  // level r: each thread's run of E; run direction = bit r of k = bit 0 of tid
  thread_sort(f, (tid & 1u) != 0);
  // The level loop stays rolled (code size); register indices inside it are
  // compile-time constants, guarded by uniform runtime conditions.
#pragma unroll 1
  for (int j = r + 1; j <= t; ++j) {
    // merge sorted blocks of 2^(j-1) into blocks of 2^j; a block is ascending
    // iff bit j of its index k is 0 (always ascending at the last level)
    const bool desc_blk = (j < t) && (((tid >> (j - r)) & 1u) != 0);
    int top_lane_bit = j - 1;
    if (j - 1 >= r + 5) {
      // bits j-1 .. t-r are warp bits in BLK but register bits in STR
      blk_to_str<NT>(f, sm, plane);
      // direction of register e in STR: bit j of k = e*NT + tid
      uint32_t dmask = 0;
      if (j < t) {
        if (j >= t - r) {
          constexpr uint32_t kBitPattern[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u,
                                               0xFF00FF00u, 0xFFFF0000u};
          dmask = kBitPattern[j - (t - r)];
        } else {
          dmask = ((tid >> j) & 1u) ? 0xFFFFFFFFu : 0u;
        }
      }
      const int rb_top = j - 1 - (t - r);
#pragma unroll
      for (int rb = r - 1; rb >= 0; --rb) {
        if (rb > rb_top) continue;
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (!(e & (1 << rb))) ce(f, e, e | (1 << rb), ((dmask >> e) & 1u) != 0);
      }
      str_to_blk<NT>(f, sm, plane);
      top_lane_bit = t - r - 1;
    }
#pragma unroll 1
    for (int b = top_lane_bit; b >= r; --b) shfl_stage(f, 1 << (b - r), desc_blk);
#pragma unroll
    for (int rb = r - 1; rb >= 0; --rb) {
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (!(e & (1 << rb))) ce(f, e, e | (1 << rb), desc_blk);
    }
  }
}

template <typename K, int V> struct VecOf;
template <> struct VecOf<uint32_t, 4> { using T = uint4; };
template <> struct VecOf<uint64_t, 2> { using T = ulonglong2; };
template <int V> struct ValVec;
template <> struct ValVec<4> { using T = uint4; };
template <> struct ValVec<2> { using T = uint2; };

template <typename K, bool PAIRS, int E, int NT>
__global__ void __launch_bounds__(NT) block_sort_kernel(const BlockSortArgs a) {
  constexpr int T = E * NT;
  constexpr int V = 16 / sizeof(K);  // keys per 16-byte vector
  using KV = typename VecOf<K, V>::T;
  using VV = typename ValVec<V>::T;
  extern __shared__ __align__(16) uint32_t sm[];
  constexpr uint32_t plane = padded_words(T);

  Frag<K, PAIRS, E> f;
  const uint32_t tid = threadIdx.x;
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * T;
  const uint64_t rem = a.n - base;
  const uint32_t cnt = rem < static_cast<uint64_t>(T) ? static_cast<uint32_t>(rem) : T;
  const K* kin = static_cast<const K*>(a.kin) + base;
  const uint32_t* vin = PAIRS ? a.vin + base : nullptr;

  if (cnt == T) {
#pragma unroll
    for (int q = 0; q < E / V; ++q) {
      const uint32_t pos = q * V * NT + V * tid;
      const KV kv = *reinterpret_cast<const KV*>(kin + pos);
      const K* kp = reinterpret_cast<const K*>(&kv);
#pragma unroll
      for (int c = 0; c < V; ++c) f.k[q * V + c] = map_key(kp[c], a.mode_in);
      if constexpr (PAIRS) {
        const VV vv = *reinterpret_cast<const VV*>(vin + pos);
        const uint32_t* vp = reinterpret_cast<const uint32_t*>(&vv);
#pragma unroll
        for (int c = 0; c < V; ++c) {
          f.v[q * V + c] = vp[c];
          f.ix[q * V + c] = pos + c;
        }
      }
    }
  } else {
    // ragged last tile: positions >= cnt become +inf pads that sort last
    // (their tie-break index exceeds every real one)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t pos = (e / V) * V * NT + V * tid + (e % V);
      const bool real = pos < cnt;
      f.k[e] = real ? map_key(kin[pos], a.mode_in) : KeyLimits<K>::kMax;
      if constexpr (PAIRS) {
        f.v[e] = real ? vin[pos] : 0u;
        f.ix[e] = pos;
      }
    }
  }

  block_bitonic_sort<NT>(f, sm, plane);

  K* kout = static_cast<K*>(a.kout) + base;
  uint32_t* vout = PAIRS ? a.vout + base : nullptr;
  const uint32_t p0 = tid * E;
  if (p0 + E <= cnt) {
#pragma unroll
    for (int q = 0; q < E / V; ++q) {
      KV kv;
      K* kp = reinterpret_cast<K*>(&kv);
#pragma unroll
      for (int c = 0; c < V; ++c) kp[c] = unmap_key(f.k[q * V + c], a.mode_out);
      *reinterpret_cast<KV*>(kout + p0 + q * V) = kv;
    }
    if constexpr (PAIRS) {
#pragma unroll
      for (int q = 0; q < E / 4; ++q)
        *reinterpret_cast<uint4*>(vout + p0 + 4 * q) =
            make_uint4(f.v[4 * q], f.v[4 * q + 1], f.v[4 * q + 2], f.v[4 * q + 3]);
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (p0 + e < cnt) {
        kout[p0 + e] = unmap_key(f.k[e], a.mode_out);
        if constexpr (PAIRS) vout[p0 + e] = f.v[e];
      }
    }
  }
}

// ---------------------------------------------------------------- dispatch

template <typename K, bool PAIRS, int E, int NT>
static cudaError_t launch_bs(const BlockSortArgs& a, cudaStream_t s) {
  constexpr int T = E * NT;
  constexpr int W = Frag<K, PAIRS, E>::W;
  const size_t smem = static_cast<size_t>(W) * padded_words(T) * sizeof(uint32_t);
  auto kern = block_sort_kernel<K, PAIRS, E, NT>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  const uint64_t tiles = (a.n + T - 1) / T;
  if (tiles == 0) return cudaSuccess;
  kern<<<static_cast<unsigned>(tiles), NT, smem, s>>>(a);
  return cudaGetLastError();
}

// Register budget: pairs with E = 32 would need ~100 data registers per
// thread, so only E = 16 is built for pairs.
bool block_cfg_supported(int key_bytes, bool pairs, int cfg) {
  if (cfg < 0 || cfg >= kNumBlockCfgs) return false;
  if (key_bytes != 4 && key_bytes != 8) return false;
  return !(pairs && kBlockCfgs[cfg].E > 16);
}

template <typename K, bool PAIRS>
static cudaError_t dispatch_bs(int cfg, const BlockSortArgs& a, cudaStream_t s) {
  switch (cfg) {
    case 0: return launch_bs<K, PAIRS, 16, 256>(a, s);
    case 1: return launch_bs<K, PAIRS, 16, 512>(a, s);
    case 2:
      if constexpr (!PAIRS) return launch_bs<K, PAIRS, 32, 256>(a, s);
      break;
    case 3:
      if constexpr (!PAIRS) return launch_bs<K, PAIRS, 32, 512>(a, s);
      break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_block_sort(int key_bytes, bool pairs, int cfg, const BlockSortArgs& a,
                              cudaStream_t s) {
  if (!block_cfg_supported(key_bytes, pairs, cfg)) return cudaErrorInvalidValue;
  if (key_bytes == 4)
    return pairs ? dispatch_bs<uint32_t, true>(cfg, a, s) : dispatch_bs<uint32_t, false>(cfg, a, s);
  return pairs ? dispatch_bs<uint64_t, true>(cfg, a, s) : dispatch_bs<uint64_t, false>(cfg, a, s);
}

}  // namespace bcf
