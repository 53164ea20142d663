// bcf_cps.cu -- colored prefix sums (Appendix A).
//
// Problem: elements i = 0..n-1 carry a value v[i] (u32) and a color c[i] in
// [0, d); out[i] is the sum, modulo 2^32, of the values of the elements of
// color c[i] at positions <= i (inclusive) or < i (exclusive): d independent
// prefix sums.  The paper uses it to show that shared-memory bank conflicts,
// not the asymptotic work, make the runtime grow with d (Sec. 2.2, Fig. 2),
// and removes them by giving every thread its own bank for its per-color
// counters (Appendix A).
//
// GB300 design: one pass over HBM (read v and c once, write out once).
//   * Tiles of kCpsTile = 16384 elements, one per CTA, taken in order from an
//     atomic ticket so that every tile's predecessors are already running.
//     Large tiles keep the chain across tiles short (see the look-back).
//   * Each thread owns 64 consecutive elements (the paper's "contiguous
//     chunk"), streamed in kCpsSteps steps of kCpsPerThread with the next
//     step's loads in flight.  The run is read twice -- once for the totals,
//     once for the outputs -- and the second read hits L2 (the tile was read
//     microseconds before), so HBM sees one read and one write.
//   * Per-thread, per-color sums live in a d x NT shared-memory matrix.  In
//     the conflict-free layout (the paper's) word(c, t) = c * NT + t: a warp's
//     lanes always touch 32 different banks, whatever colors they hold.  The
//     other layout, word(c, t) = t * d + c, keeps a thread's counters together
//     and is the conflicting baseline of the paper's experiment.
//   * Each warp scans whole color rows with warp shuffles (the row-wise scan
//     the paper gets by transposing the matrix), giving every thread its
//     exclusive in-tile prefix per color and every color its tile total.
//   * Across tiles: a decoupled look-back on one status word per (tile,
//     color) -- flag in the top bits, 32-bit sum below -- publishing the tile
//     total first and the inclusive prefix once known.  Every warp looks
//     back for its share of the colors, many predecessors per round (one
//     load per lane), so the walk stays short however many tiles are in
//     flight.  The wait on a predecessor is bounded by the global timer; on
//     expiry the device error word is set and the tile proceeds, so the grid
//     always finishes.
//   * A final sweep over the thread's run produces the outputs, stored with
//     32-byte vector stores.
// Colors >= d are a precondition violation: such elements contribute nothing,
// their output is 0 and the device error word gets kErrBadColor.  Inside the
// library the same kernel also runs as a plain prefix sum (no color array,
// d = 1), e.g. over the pivot-bucket sort's bucket counts.
#include <cuda_runtime.h>

#include "bcf_device.cuh"
#include "bcf_internal.h"

namespace bcf {

namespace {

constexpr int NT = kCpsThreads;
constexpr int E = kCpsPerThread;
constexpr unsigned long long kFlagAggregate = 1ull << 62;
constexpr unsigned long long kFlagInclusive = 2ull << 62;

template <bool BANKED>
__device__ __forceinline__ uint32_t word_of(uint32_t c, uint32_t t, uint32_t d) {
  return BANKED ? c * NT + t : t * d + c;
}

// The status word holds flag and sum together and carries no other data, so
// relaxed (unordered) single-copy-atomic 64-bit accesses suffice.
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void ld_global_32B(const uint32_t* p, uint32_t* x) {
  asm volatile("ld.global.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]),
                 "=r"(x[6]), "=r"(x[7])
               : "l"(p));
}

// Padded index of a per-color array read by lanes holding arbitrary colors:
// colors c and c + 32 land in different banks.
__device__ __forceinline__ uint32_t cpad(uint32_t c) { return c + (c >> 5); }

// One step of one thread: E values and E colors packed 4 per word.
struct StepRegs {
  uint32_t v[E];
  uint32_t cw[E / 4];
};

// Loads step `step` of this thread's run: elements [p, p + E) of the tile
// with p = tid * E * kSteps + step * E; `cnt` elements of the tile are real.
template <bool FULL>
__device__ __forceinline__ void load_step(const CpsArgs& a, uint64_t base, uint32_t cnt,
                                          uint32_t p, StepRegs& r) {
  if (FULL || p + E <= cnt) {
    const uint32_t* vp = a.values + base + p;
    if (is_aligned32(a.values)) {
      ld_global_32B(vp, r.v);
      ld_global_32B(vp + 8, r.v + 8);
    } else {
#pragma unroll
      for (int q = 0; q < E / 4; ++q) {
        const uint4 x = *reinterpret_cast<const uint4*>(vp + 4 * q);
        r.v[4 * q] = x.x; r.v[4 * q + 1] = x.y; r.v[4 * q + 2] = x.z; r.v[4 * q + 3] = x.w;
      }
    }
    if (a.colors) {
      const uint4 c4 = *reinterpret_cast<const uint4*>(a.colors + base + p);
      r.cw[0] = c4.x; r.cw[1] = c4.y; r.cw[2] = c4.z; r.cw[3] = c4.w;
    } else {
#pragma unroll
      for (int q = 0; q < E / 4; ++q) r.cw[q] = 0u;
    }
  } else {
#pragma unroll
    for (int q = 0; q < E / 4; ++q) r.cw[q] = 0u;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const bool real = p + e < cnt;
      r.v[e] = real ? a.values[base + p + e] : 0u;
      const uint32_t c = (real && a.colors) ? a.colors[base + p + e] : 0u;
      r.cw[e / 4] |= c << (8 * (e % 4));
    }
  }
}

__device__ __forceinline__ uint32_t color_of(const StepRegs& r, int e) {
  return (r.cw[e / 4] >> (8 * (e % 4))) & 0xFFu;
}

// One tile.  FULL: all kCpsTile elements are real (every tile but a ragged
// last one), so no element needs a bounds check.
template <bool BANKED, int kLookbackLoads, bool FULL>
__device__ __forceinline__ void cps_tile(const CpsArgs& a, uint32_t* sm, uint64_t tile,
                                         uint32_t cnt) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t d = a.d;
  uint32_t* mat = sm;                      // d * NT counters
  uint32_t* s_excl = sm + d * NT;          // tile-exclusive prefix per color (padded)
  uint32_t* s_agg = s_excl + cpad(d) + 1;  // tile total per color (padded)
  const uint64_t base = tile * kCpsTile;
  const uint32_t p0 = tid * E * kCpsSteps;  // this thread's run of E * kCpsSteps elements

  // ---- phase 1: per-thread totals per color, in the thread's own bank; the
  // next step's loads are in flight while one step is accumulated
  bool bad = false;
  StepRegs r[2];
  load_step<FULL>(a, base, cnt, p0, r[0]);
#pragma unroll
  for (int st = 0; st < kCpsSteps; ++st) {
    if (st + 1 < kCpsSteps) load_step<FULL>(a, base, cnt, p0 + (st + 1) * E, r[(st + 1) & 1]);
    const StepRegs& x = r[st & 1];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t c = color_of(x, e);
      const bool real = FULL || p0 + st * E + e < cnt;
      // a shared-memory reduction: no dependence between consecutive elements
      // (each thread owns its counters, so nothing contends)
      if (real && c < d) atomicAdd(mat + word_of<BANKED>(c, tid, d), x.v[e]);
      bad |= real && c >= d;
    }
  }
  if (bad) atomicOr(a.err, kErrBadColor);
  // the second sweep re-reads the run (from L2: the tile was just read); its
  // first step is issued now, ahead of the scan and the look-back
  load_step<FULL>(a, base, cnt, p0, r[0]);
  __syncthreads();

  // ---- phase 2: scan every color row over the threads; publish tile totals
  for (uint32_t c = warp; c < d; c += NT / 32) {
    uint32_t carry = 0;
#pragma unroll
    for (int j = 0; j < NT / 32; ++j) {
      const uint32_t w = word_of<BANKED>(c, j * 32 + lane, d);
      const uint32_t x = mat[w];
      uint32_t s = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
        if (lane >= static_cast<uint32_t>(o)) s += y;
      }
      mat[w] = carry + s - x;  // exclusive prefix of thread j*32+lane within the tile
      carry += __shfl_sync(0xFFFFFFFFu, s, 31);
    }
    if (lane == 0) {
      s_agg[cpad(c)] = carry;
      st_relaxed(a.status + tile * d + c, (tile == 0 ? kFlagInclusive : kFlagAggregate) | carry);
    }
  }
  __syncthreads();

  // ---- look-back across tiles.  Warp w serves colors c = w + 8 s; its lanes
  // form K color slots s (K = colors per warp rounded up to a power of two)
  // times J = 32 / K offsets j, and every lane loads kLookbackLoads
  // predecessors (offsets j, j + J, ...), so one round inspects a window of
  // J * kLookbackLoads predecessors of K colors with independent loads.  Per
  // slot, the nearest predecessor that has published its inclusive prefix
  // ends the walk and the totals of the nearer ones are added to it.  A slot
  // whose window holds, before that point, a predecessor that has published
  // nothing yet re-reads the window (bounded wait with back-off); a slot with
  // no inclusive prefix in its window adds every total and moves the window
  // back.  Throughput of the chain across tiles is one window per L2 round
  // trip, hence the wide windows.
  {
    constexpr uint32_t kWarps = NT / 32;
        const uint32_t ncol = d > warp ? (d - warp + kWarps - 1) / kWarps : 0u;
    if (ncol > 0) {
      uint32_t K = 1;
      while (K < ncol) K <<= 1;
      const uint32_t J = 32u / K;
      const uint32_t slot = lane & (K - 1u), j = lane / K;
      const uint32_t c = warp + kWarps * slot;
      uint32_t slot_lanes = 0;  // lanes of this slot: slot, slot + K, ...
      for (uint32_t l = slot; l < 32; l += K) slot_lanes |= 1u << l;
      bool done = slot >= ncol || tile == 0;
      uint32_t excl = 0;
      int64_t top = static_cast<int64_t>(tile) - 1;  // predecessor at window offset 0
      uint64_t t0 = 0;
      uint32_t backoff = 32;
      while (true) {
        if (__all_sync(0xFFFFFFFFu, done)) break;
        unsigned long long st[kLookbackLoads];
#pragma unroll
        for (int q = 0; q < kLookbackLoads; ++q) {
          st[q] = 0;
          if (!done) {
            const int64_t p = top - static_cast<int64_t>(j + q * J);
            st[q] = p >= 0 ? ld_relaxed(a.status + static_cast<uint64_t>(p) * d + c)
                           : kFlagInclusive;  // before tile 0: an inclusive prefix of 0
          }
        }
        // walk the sub-windows from the nearest: add totals until an inclusive
        // prefix; stop (and wait) at a predecessor that has published nothing
        bool found = false, wait = false;
        uint32_t x = 0;
#pragma unroll
        for (int q = 0; q < kLookbackLoads; ++q) {
          const unsigned long long flag = st[q] & (3ull << 62);
          const uint32_t incl = __ballot_sync(0xFFFFFFFFu, !done && flag == kFlagInclusive);
          const uint32_t none = __ballot_sync(0xFFFFFFFFu, !done && flag == 0);
          const uint32_t mine = incl & slot_lanes;
          const uint32_t last = mine ? __ffs(mine) - 1u : 31u;  // nearest inclusive here
          const uint32_t upto = last >= 31u ? 0xFFFFFFFFu : ((2u << last) - 1u);
          const bool live = !done && !found && !wait;
          if (live && (none & slot_lanes & upto) != 0) wait = true;
          uint32_t y = (live && !wait && lane <= last) ? static_cast<uint32_t>(st[q]) : 0u;
          for (uint32_t o = K; o < 32; o <<= 1) y += __shfl_xor_sync(0xFFFFFFFFu, y, o);
          if (live && !wait) {
            x += y;
            if (mine) found = true;
          }
        }
        if (!done) {
          if (wait) {
            const uint64_t now = globaltimer_ns();
            if (t0 == 0) {
              t0 = now;
            } else if (now - t0 > a.wait_ns) {
              if (j == 0) atomicOr(a.err, kErrLookbackTimeout);
              done = true;
            }
            if (!done) {
              __nanosleep(backoff);
              backoff = backoff < 256 ? 2 * backoff : 256;
            }
          } else {
            t0 = 0;
            backoff = 32;
            excl += x;
            if (found) done = true;
            else top -= static_cast<int64_t>(J) * kLookbackLoads;
          }
        }
      }
      if (j == 0 && slot < ncol) {
        if (tile > 0)
          st_relaxed(a.status + tile * d + c, kFlagInclusive | (excl + s_agg[cpad(c)]));
        s_excl[cpad(c)] = excl;
      }
    }
  }
  __syncthreads();

  // ---- phase 3: running sums through the thread's run, step by step
#pragma unroll
  for (int st = 0; st < kCpsSteps; ++st) {
    if (st + 1 < kCpsSteps) load_step<FULL>(a, base, cnt, p0 + (st + 1) * E, r[(st + 1) & 1]);
    StepRegs& x = r[st & 1];
    const uint32_t p = p0 + st * E;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t c = color_of(x, e);
      uint32_t o = 0u;
      if ((FULL || p + e < cnt) && c < d) {
        // fetch-and-add returns the running sum before this element; the adds
        // of consecutive elements are issued back to back
        const uint32_t before = atomicAdd(mat + word_of<BANKED>(c, tid, d), x.v[e]);
        o = (a.exclusive ? before : before + x.v[e]) + s_excl[cpad(c)];
      }
      x.v[e] = o;
    }
    uint32_t* op = a.out + base + p;
    if (FULL || p + E <= cnt) {
      store_run<E>(op, x.v, is_aligned32(a.out));
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (p + e < cnt) op[e] = x.v[e];
    }
  }
}

// Four CTAs per SM (64 registers a thread; the banked layout spills a few
// words to local memory).  With the full-tile path this measured about 6 %
// faster than three CTAs at 80 registers for d <= 16 and the same at d = 64,
// where shared memory allows three CTAs anyway.
template <bool BANKED, int kLookbackLoads>
__global__ void __launch_bounds__(NT, 4) cps_kernel(const CpsArgs a) {
  extern __shared__ uint32_t sm[];
  __shared__ uint32_t s_tile;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(a.counter, 1u);
  for (uint32_t i = tid; i < a.d * NT; i += NT) sm[i] = 0u;
  __syncthreads();
  const uint64_t tile = s_tile;
  const uint64_t rem = a.n - tile * kCpsTile;
  if (rem >= static_cast<uint64_t>(kCpsTile))
    cps_tile<BANKED, kLookbackLoads, true>(a, sm, tile, kCpsTile);
  else
    cps_tile<BANKED, kLookbackLoads, false>(a, sm, tile, static_cast<uint32_t>(rem));
}

}  // namespace

size_t cps_smem_bytes(uint32_t d) {
  // matrix, then the two padded per-color arrays
  return (static_cast<size_t>(d) * NT + 2 * (d + (d >> 5) + 2)) * sizeof(uint32_t);
}

template <bool BANKED, int LB>
static cudaError_t launch_cps_t(const CpsArgs& a, size_t smem, cudaStream_t s) {
  auto kern = cps_kernel<BANKED, LB>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  CpsArgs b = a;
  b.wait_ns = wait_limit_ns();
  kern<<<static_cast<unsigned>(a.ntiles), NT, smem, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_cps(const CpsArgs& a, int layout, cudaStream_t s) {
  if (a.ntiles == 0) return cudaSuccess;
  if (a.d < 1 || a.d > kCpsMaxColors || a.ntiles > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  const size_t smem = cps_smem_bytes(a.d);
  return layout == 0 ? launch_cps_t<true, 1>(a, smem, s) : launch_cps_t<false, 1>(a, smem, s);
}

}  // namespace bcf
