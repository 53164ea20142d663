// bcf_block_sort.cuh -- the base case: every tile of T consecutive keys (plus
// payloads) sorted inside one CTA without a single shared-memory bank
// conflict (Sec. 3.1, "Base case"; Algorithms 1, 2 and 5).
//
// The paper sorts a w x w matrix in shared memory with ShearSort: register
// Batcher networks on rows and columns, transposes in between, and shifted
// diagonals so no transpose conflicts.  On sm_103a the same principles are
// kept -- data-oblivious register networks, one thread per row/column of a
// skewed shared-memory matrix -- but ShearSort's O(log w) row/column rounds
// are replaced by a bitonic sort whose cross-thread stages all go through
// conflict-free padded transposes, which needs far fewer compare-exchanges
// per key for tiles of 4K-16K keys.
//
//   1. coalesced 128-bit loads straight into registers (each thread takes V
//      consecutive keys from every NT*V-key stripe); keys are mapped to
//      unsigned order (the key type's map, then descending);
//   2. Batcher odd-even merge sort of the thread's E registers;
//   3. bitonic merge levels j = r+1 .. t: every stage is an ascending
//      register compare-exchange in one of three layouts (BLK / MID / STR),
//      joined by conflict-free padded transposes; the bitonic "flip" of each
//      level is folded into the transpose's read addresses;
//   4. 32-byte stores of the thread's E consecutive outputs.
// The kernel is instantiated per key type in bcf_block_sort_*.cu (separate
// translation units, compiled in parallel); bcf_block_sort.cu dispatches.
// Pairs carry a tie-break index (input position in the tile) so that the
// result is the stable order; their payloads do not travel through the
// network: they wait in a padded shared-memory plane, loaded with the keys,
// and each output's payload is read from it by that position.
#pragma once

#include <cuda_runtime.h>

#include "bcf_device.cuh"
#include "bcf_internal.h"

namespace bcf {

// MAP: the key map is applied on load / undone on store (runtime mode); when
// false the kernel carries no map code at all (intermediate passes).
template <typename K, bool PAIRS, int E, int NT, bool MAP>
__global__ void __launch_bounds__(NT) block_sort_kernel(const BlockSortArgs a) {
  constexpr int T = E * NT;
  constexpr int V = 16 / sizeof(K);  // keys per 16-byte vector
  using KV = typename VecOf<K, V>::T;
  using VV = typename ValVec<V>::T;
  extern __shared__ __align__(16) uint32_t sm[];

  // with payloads the network sorts (key, position) only: the tile's payloads
  // wait in their own padded plane behind the network's planes, and each
  // output's payload is read from there by its position once the tile is
  // sorted (the network's barriers order the plane's writes before the reads)
  Frag<K, PAIRS, E, /*VALS=*/false> f;
  uint32_t* sv = sm + Frag<K, PAIRS, E, false>::W * padded_words(T);
  // keys-only 32-bit tiles move the BLK stages' maxima to the FMA pipe (the
  // network is bound by the ALU pipe: measured 1.87 vs 1.98 ms at 2^28 keys;
  // the multiplier is read before the tile's loads, which measured faster than
  // reading it just before the network)
  f.one = g_unit_multiplier;
  const uint32_t tid = threadIdx.x;
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * T;
  const uint64_t rem = a.n - base;
  const uint32_t cnt = rem < static_cast<uint64_t>(T) ? static_cast<uint32_t>(rem) : T;
  const K* kin = static_cast<const K*>(a.kin) + base;
  const uint32_t* vin = PAIRS ? a.vin + base : nullptr;
  const int mode_in = MAP ? a.mode_in : 0;
  const int mode_out = MAP ? a.mode_out : 0;

  if (cnt == T) {
#pragma unroll
    for (int q = 0; q < E / V; ++q) {
      const uint32_t pos = q * V * NT + V * tid;
      const KV kv = *reinterpret_cast<const KV*>(kin + pos);
      const K* kp = reinterpret_cast<const K*>(&kv);
#pragma unroll
      for (int c = 0; c < V; ++c) f.k[q * V + c] = MAP ? map_key(kp[c], mode_in) : kp[c];
      if constexpr (PAIRS) {
        const VV vv = *reinterpret_cast<const VV*>(vin + pos);
        const uint32_t* vp = reinterpret_cast<const uint32_t*>(&vv);
#pragma unroll
        for (int c = 0; c < V; ++c) {
          f.ix[q * V + c] = pos + c;
          sv[pos + c + ((pos + c) >> 5)] = vp[c];
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
      K x = KeyLimits<K>::kMax;
      if (real) x = MAP ? map_key(kin[pos], mode_in) : kin[pos];
      f.k[e] = x;
      if constexpr (PAIRS) {
        f.ix[e] = pos;
        sv[pos + (pos >> 5)] = real ? vin[pos] : 0u;
      }
    }
  }

  block_sort_tile<NT, CeForms<K, PAIRS>::kBlockBlk, CeForms<K, PAIRS>::kBlockOth>(f, sm);

  K* kout = static_cast<K*>(a.kout) + base;
  uint32_t* vout = PAIRS ? a.vout + base : nullptr;
  const uint32_t p0 = tid * E;
  // sample of the sorted tile for the next pass's merge-path search (mapped keys)
  static_assert(kSampleStride % E == 0 && T % kSampleStride == 0, "sample stride");
  if (a.samples && (p0 % kSampleStride) == 0 && p0 < cnt)
    static_cast<K*>(a.samples)[(base + p0) / kSampleStride] = f.k[0];
  // payloads by tile position from the payload plane
  uint32_t vg[PAIRS ? E : 1];
  if constexpr (PAIRS) {
#pragma unroll
    for (int e = 0; e < E; ++e) vg[e] = sv[f.ix[e] + (f.ix[e] >> 5)];
  }
  if (p0 + E <= cnt) {
    // base and p0 are multiples of 32 bytes: the base pointers decide alignment
    if constexpr (MAP) {
#pragma unroll
      for (int e = 0; e < E; ++e) f.k[e] = unmap_key(f.k[e], mode_out);  // last use of f.k
    }
    store_run<E>(kout + p0, f.k, is_aligned32(a.kout));
    if constexpr (PAIRS) store_run<E>(vout + p0, vg, is_aligned32(a.vout));
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (p0 + e < cnt) {
        kout[p0 + e] = MAP ? unmap_key(f.k[e], mode_out) : f.k[e];
        if constexpr (PAIRS) vout[p0 + e] = vg[e];
      }
    }
  }
}

// ---------------------------------------------------------------- dispatch

template <typename K, bool PAIRS, int E, int NT>
static cudaError_t launch_bs(const BlockSortArgs& a, cudaStream_t s) {
  constexpr int T = E * NT;
  // the network's planes, plus the payload plane with payloads
  constexpr int W = Frag<K, PAIRS, E, /*VALS=*/false>::W + (PAIRS ? 1 : 0);
  const size_t need = static_cast<size_t>(W) * padded_words(T) * sizeof(uint32_t);
  const size_t smem = need > smem_floor_bytes() ? need : smem_floor_bytes();
  const uint64_t tiles = (a.n + T - 1) / T;
  if (tiles == 0) return cudaSuccess;
  const bool map = (a.mode_in | a.mode_out) != 0;
  auto kern = map ? block_sort_kernel<K, PAIRS, E, NT, true>
                  : block_sort_kernel<K, PAIRS, E, NT, false>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  kern<<<static_cast<unsigned>(tiles), NT, smem, s>>>(a);
  return cudaGetLastError();
}

// Launch the block sort of configuration `cfg` for key type K.
template <typename K, bool PAIRS>
cudaError_t launch_block_sort_typed(int cfg, const BlockSortArgs& a, cudaStream_t s) {
  switch (cfg) {
    case 0: return launch_bs<K, PAIRS, 16, 256>(a, s);
    case 1:
      if constexpr (!(PAIRS && sizeof(K) == 8)) return launch_bs<K, PAIRS, 32, 256>(a, s);
      break;
    case 2:
      if constexpr (!(PAIRS && sizeof(K) == 8)) return launch_bs<K, PAIRS, 32, 512>(a, s);
      break;
    case 3:
      if constexpr (!(PAIRS && sizeof(K) == 8)) return launch_bs<K, PAIRS, 32, 128>(a, s);
      break;
    case 4:
      if constexpr (!PAIRS && sizeof(K) == 4) return launch_bs<K, PAIRS, 32, 1024>(a, s);
      break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace bcf
