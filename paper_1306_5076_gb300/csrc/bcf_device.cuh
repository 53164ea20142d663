// bcf_device.cuh -- device building blocks shared by the block sort, the merge
// pass and the segmented sort.
//
// Data model.  A CTA holds a logical array X[0, 2^t) of elements spread over
// its threads' registers, E = 2^r elements per thread.  Two register layouts
// are used (the paper's row/column views of shared memory, Sec. 2.1, taken to
// registers):
//   BLK: thread tid holds X[tid * E + e]        (register bits = k bits [0, r))
//   STR: thread tid holds X[e * NT + tid]       (register bits = k bits [t-r, t))
// A bitonic stage on bit b pairs X[k] with X[k ^ 2^b].  It is a register
// compare-exchange when b is a register bit of the current layout, a warp
// shuffle when b is a lane bit of BLK (bits [r, r+5)), and otherwise needs a
// switch of layout through shared memory.  With t <= 2r + 5 the two layouts
// cover every bit, so every cross-thread step is either a shuffle or one
// transpose through shared memory.
//
// Bank conflicts.  The transposes go through shared memory in 32-bit planes
// (one plane per 32-bit word of an element) with one pad word after every 32
// words: physical word = k + (k >> 5).  In STR a warp touches 32 consecutive
// k, i.e. 32 distinct banks.  In BLK lane l touches k = l*E + e; its bank is
// (l*E + e + floor(l*E / 32)) mod 32, which is a bijection of l for every
// power of two E <= 32 -- the skew the paper obtains with shifted diagonals
// (Sec. 3.3, Algorithm 2), obtained here by padding.  So every shared-memory
// access of the sorting network is conflict-free.
#pragma once

#include <cstdint>
#include <type_traits>

namespace bcf {

// ---------------------------------------------------------------- constants

constexpr uint32_t kErrTmaTimeout = 1u;

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

// ---------------------------------------------------------------- key maps
// Order-preserving maps from key bits to unsigned integers, applied when a
// key is first loaded and undone when it is last stored.
//   mode bit 0: IEEE 754 totalOrder (f32 on 32-bit keys, f64 on 64-bit keys):
//               a negative-signed pattern has all its bits inverted, a
//               positive-signed one its sign bit set, so that unsigned order
//               equals totalOrder;
//   mode bit 2: two's-complement order (i32 / i64): the sign bit is flipped;
//   mode bit 1: descending (bitwise NOT, after the type's map).
// Each map is a bijection and unmap inverts it exactly, so keys come back
// bit-for-bit.

template <typename U>
__device__ __forceinline__ U map_key(U u, int mode) {
  constexpr int kTop = 8 * sizeof(U) - 1;
  constexpr U kSign = U(1) << kTop;
  using S = typename std::conditional<sizeof(U) == 4, int32_t, int64_t>::type;
  if (mode & 1) u ^= U(S(u) >> kTop) | kSign;
  if (mode & 4) u ^= kSign;
  if (mode & 2) u = ~u;
  return u;
}
template <typename U>
__device__ __forceinline__ U unmap_key(U m, int mode) {
  constexpr int kTop = 8 * sizeof(U) - 1;
  constexpr U kSign = U(1) << kTop;
  using S = typename std::conditional<sizeof(U) == 4, int32_t, int64_t>::type;
  if (mode & 2) m = ~m;
  if (mode & 4) m ^= kSign;
  if (mode & 1) m ^= U(~U(S(m) >> kTop)) | kSign;
  return m;
}

template <typename K> struct KeyLimits;
template <> struct KeyLimits<uint32_t> {
  static constexpr uint32_t kMin = 0u, kMax = 0xFFFFFFFFu;
};
template <> struct KeyLimits<uint64_t> {
  static constexpr uint64_t kMin = 0ull, kMax = ~0ull;
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization (launch_chained) is scheduled as soon as the kernel ahead of
// it in the stream has run its last CTA, without the full kernel boundary in
// between.  pdl_wait() blocks until that kernel has completed and its memory
// operations are visible (a no-op for a normal launch), so it precedes every
// global access of the waiting kernel: reads of what the predecessor wrote
// and writes over what it reads alike.  No kernel here releases its
// dependents early (griddepcontrol.launch_dependents): CTAs of the next
// kernel resident and waiting while a merge pass's last CTAs ran made the
// u32 + u32 sort at 2^28 2.6 % slower (17.91 against 17.45 ms).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the barrier, at most limit_ns.  On expiry the
// error word gets `code` and false is returned.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* err,
                                                  uint32_t code, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) {
      if (err) atomicOr(err, code);
      return false;
    }
  }
  return true;
}
// One bulk (non-tensor) global -> shared copy completing on `bar`.  dst, src
// and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Shared loads issued only by lanes whose predicate is set; the others keep
// `dflt`.  Two such loads with disjoint predicates stay two separate
// requests, so lanes reading two different arrays never share a wavefront.
__device__ __forceinline__ uint32_t lds_pred(const uint32_t* p, bool pred, uint32_t dflt) {
  uint32_t v = dflt;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.shared.b32 %0, [%1];\n\t}"
      : "+r"(v)
      : "r"(smem_u32(p)), "r"((uint32_t)pred)
      : "memory");
  return v;
}
__device__ __forceinline__ uint64_t lds_pred(const uint64_t* p, bool pred, uint64_t dflt) {
  uint64_t v = dflt;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.shared.b64 %0, [%1];\n\t}"
      : "+l"(v)
      : "r"(smem_u32(p)), "r"((uint32_t)pred)
      : "memory");
  return v;
}

// Shared store issued only by lanes whose predicate is set (one instruction of
// its own: lanes storing to two different arrays through two such calls never
// share a request).
__device__ __forceinline__ void sts_pred(uint32_t* p, bool pred, uint32_t v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.b32 [%0], %1;\n\t}"
               ::"r"(smem_u32(p)), "r"(v), "r"((uint32_t)pred)
               : "memory");
}
__device__ __forceinline__ void sts_pred(uint64_t* p, bool pred, uint64_t v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.b64 [%0], %1;\n\t}"
               ::"r"(smem_u32(p)), "l"(v), "r"((uint32_t)pred)
               : "memory");
}

// 32-byte global stores (sm_100 and later): each thread writes one whole
// 32-byte sector, so a warp storing its threads' consecutive runs touches
// full sectors only, with half the store instructions of 16-byte vectors.
// `p` must be 32-byte aligned.
__device__ __forceinline__ void st_global_32B(uint32_t* p, const uint32_t* x) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(x[0]),
               "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7])
               : "memory");
}
__device__ __forceinline__ void st_global_32B(uint64_t* p, const uint64_t* x) {
  asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(x[0]), "l"(x[1]),
               "l"(x[2]), "l"(x[3])
               : "memory");
}

// 16-byte vectors of V keys, and of the V payloads that go with them.
template <typename K, int V> struct VecOf;
template <> struct VecOf<uint32_t, 4> { using T = uint4; };
template <> struct VecOf<uint64_t, 2> { using T = ulonglong2; };
template <int V> struct ValVec;
template <> struct ValVec<4> { using T = uint4; };
template <> struct ValVec<2> { using T = uint2; };

// Stores E consecutive elements x[0..E) of one thread at p (E * sizeof(K) a
// multiple of 32): 32-byte stores when p is 32-byte aligned, else 16-byte.
template <int E, typename K>
__device__ __forceinline__ void store_run(K* p, const K* x, bool aligned32) {
  constexpr int V32 = 32 / sizeof(K), V16 = 16 / sizeof(K);
  static_assert((E * sizeof(K)) % 32 == 0, "run must be whole 32-byte sectors");
  if (aligned32) {
#pragma unroll
    for (int q = 0; q < E / V32; ++q) st_global_32B(p + q * V32, x + q * V32);
  } else {
    using KV = typename std::conditional<sizeof(K) == 4, uint4, ulonglong2>::type;
#pragma unroll
    for (int q = 0; q < E / V16; ++q) {
      KV kv;
      K* kp = reinterpret_cast<K*>(&kv);
#pragma unroll
      for (int c = 0; c < V16; ++c) kp[c] = x[q * V16 + c];
      *reinterpret_cast<KV*>(p + q * V16) = kv;
    }
  }
}

__device__ __forceinline__ bool is_aligned32(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 31u) == 0;
}

// ---------------------------------------------------------------- elements

// Padded shared-memory index of logical word k (one pad word per 32 words).
__device__ __forceinline__ uint32_t pad32(uint32_t k) { return k + (k >> 5); }
__host__ __device__ constexpr uint32_t padded_words(uint32_t n) { return n + n / 32; }

// Register fragment: E elements per thread.  PAIRS carries a tie-break index
// (the element's rank in the stable input order), because bitonic networks
// are not stable on their own, and -- unless VALS is false -- the u32
// payload.  (A merge can leave the payloads out of the network and fetch each
// output's payload by its rank afterwards.)
template <typename K, bool PAIRS, int E, bool VALS = PAIRS>
struct Frag {
  static constexpr int KW = sizeof(K) / 4;                        // 32-bit words per key
  static constexpr int W = KW + (PAIRS ? (VALS ? 2 : 1) : 0);     // 32-bit planes per element
  K k[E];
  uint32_t ix[PAIRS ? E : 1];
  uint32_t v[PAIRS && VALS ? E : 1];
  uint32_t one;  // the multiplier of the FMA-pipe maximum (see ce()); set by kernels that use it

  __device__ __forceinline__ void put(uint32_t* sm, uint32_t plane, int e, uint32_t a) const {
    sm[a] = static_cast<uint32_t>(k[e]);
    if constexpr (KW == 2) sm[plane + a] = static_cast<uint32_t>(static_cast<uint64_t>(k[e]) >> 32);
    if constexpr (PAIRS) sm[KW * plane + a] = ix[e];
    if constexpr (PAIRS && VALS) sm[(KW + 1) * plane + a] = v[e];
  }
  __device__ __forceinline__ void get(const uint32_t* sm, uint32_t plane, int e, uint32_t a) {
    if constexpr (KW == 2)
      k[e] = static_cast<K>(sm[a]) | (static_cast<K>(sm[plane + a]) << 32);
    else
      k[e] = static_cast<K>(sm[a]);
    if constexpr (PAIRS) ix[e] = sm[KW * plane + a];
    if constexpr (PAIRS && VALS) v[e] = sm[(KW + 1) * plane + a];
  }
};

// Strict "x after y" in (key, tie-break index) order.
template <typename K>
__device__ __forceinline__ bool after(K kx, uint32_t ix, K ky, uint32_t iy) {
  if constexpr (sizeof(K) == 4) {
    const uint64_t x = (static_cast<uint64_t>(kx) << 32) | ix;
    const uint64_t y = (static_cast<uint64_t>(ky) << 32) | iy;
    return x > y;
  } else {
    // (key, index) as one 96-bit number: y - x with a borrow chain over the
    // three words borrows exactly when x > y
    uint32_t r;
    asm("{\n\t.reg .u32 t;\n\t"
        "sub.cc.u32 t, %1, %2;\n\t"
        "subc.cc.u32 t, %3, %4;\n\t"
        "subc.cc.u32 t, %5, %6;\n\t"
        "subc.u32 %0, 0, 0;\n\t}"
        : "=r"(r)
        : "r"(iy), "r"(ix), "r"(static_cast<uint32_t>(ky)), "r"(static_cast<uint32_t>(kx)),
          "r"(static_cast<uint32_t>(static_cast<uint64_t>(ky) >> 32)),
          "r"(static_cast<uint32_t>(static_cast<uint64_t>(kx) >> 32)));
    return r != 0;
  }
}

// A 1 that the compiler cannot fold away (it could be written from the host),
// read once per thread into Frag::one.
static __device__ uint32_t g_unit_multiplier = 1;

// Compare-exchange forms.  The networks' integer minima, maxima, comparisons
// and selects run on the ALU pipe, which takes them at half the issue rate;
// the FMA pipe, which runs integer multiply-adds at the full rate, is idle.
// The forms below move work there (with a multiplier of Frag::one); all are
// exact in modular arithmetic.
//   kFmaKeys    (32-bit keys, no payloads): the maximum is x * 1 + y - min(x, y),
//               two multiply-adds instead of a second min / max;
//   kFmaWord(w) (every other kind of element): after the one comparison that
//               decides the swap, word w is swapped as x' = x + s (y - x),
//               y' = x + y - x' with s in {0, 1} -- four multiply-adds instead
//               of two selects.  Words: 0 the key (its low half for 64-bit
//               keys), 1 the high half of a 64-bit key, 2 the tie-break index,
//               3 the payload.
// Which words take the FMA form is chosen per kernel and element kind
// (CeForms below): the best split balances the two pipes against the issue
// rate.
enum : int { kFmaKeys = 1 };
__host__ __device__ constexpr int kFmaWord(int w) { return 1 << (4 + w); }

// x' = x + s (y - x), y' = x + y - x' on the FMA pipe (s = 0 or 1 = one).
__device__ __forceinline__ void fma_swap(uint32_t& xr, uint32_t& yr, uint32_t s, uint32_t one) {
  const uint32_t x = xr, y = yr, neg = 0u - one;
  uint32_t d, nx, t, ny;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(neg), "r"(y));    // y - x
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(nx) : "r"(s), "r"(d), "r"(x));     // x + s(y - x)
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(t) : "r"(x), "r"(one), "r"(y));    // x + y
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(ny) : "r"(nx), "r"(neg), "r"(t));  // x + y - x'
  xr = nx;
  yr = ny;
}
__device__ __forceinline__ void sel_swap(uint32_t& xr, uint32_t& yr, bool sw) {
  const uint32_t x = xr, y = yr;
  xr = sw ? y : x;
  yr = sw ? x : y;
}

// Compare-exchange registers a < b: ascending puts the smaller element in a.
template <typename K, bool PAIRS, int E, bool VALS>
__device__ __forceinline__ void ce(Frag<K, PAIRS, E, VALS>& f, int a, int b, bool desc,
                                   int fma = 0) {
  if constexpr (!PAIRS && sizeof(K) == 4) {
    const uint32_t x = static_cast<uint32_t>(f.k[a]), y = static_cast<uint32_t>(f.k[b]);
    const uint32_t lo = x < y ? x : y;
    uint32_t hi;
    if (fma & kFmaKeys) {
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(hi) : "r"(x), "r"(f.one), "r"(y));
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(hi) : "r"(lo), "r"(0u - f.one), "r"(hi));
    } else {
      hi = x < y ? y : x;
    }
    f.k[a] = static_cast<K>(desc ? hi : lo);
    f.k[b] = static_cast<K>(desc ? lo : hi);
  } else if (!PAIRS && (fma & (kFmaWord(0) | kFmaWord(1))) == 0) {
    // 64-bit keys without payloads: a 64-bit minimum and maximum (measured
    // 13 % faster in the block sort than one comparison and four selects)
    const K x = f.k[a], y = f.k[b];
    const K lo = x < y ? x : y, hi = x < y ? y : x;
    f.k[a] = desc ? hi : lo;
    f.k[b] = desc ? lo : hi;
  } else {
    bool sw;  // a and b trade places
    if constexpr (PAIRS)
      sw = after(f.k[a], f.ix[a], f.k[b], f.ix[b]) != desc;
    else
      sw = (f.k[a] > f.k[b]) != desc;
    const uint32_t s = sw ? f.one : 0u;
    const auto word = [&](uint32_t& xr, uint32_t& yr, int w) {
      if (fma & kFmaWord(w))
        fma_swap(xr, yr, s, f.one);
      else
        sel_swap(xr, yr, sw);
    };
    if constexpr (sizeof(K) == 4) {
      uint32_t ka = static_cast<uint32_t>(f.k[a]), kb = static_cast<uint32_t>(f.k[b]);
      word(ka, kb, 0);
      f.k[a] = static_cast<K>(ka);
      f.k[b] = static_cast<K>(kb);
    } else {
      const uint64_t xa = static_cast<uint64_t>(f.k[a]), xb = static_cast<uint64_t>(f.k[b]);
      uint32_t la = static_cast<uint32_t>(xa), lb = static_cast<uint32_t>(xb);
      uint32_t ha = static_cast<uint32_t>(xa >> 32), hb = static_cast<uint32_t>(xb >> 32);
      word(la, lb, 0);
      word(ha, hb, 1);
      f.k[a] = static_cast<K>(la | (static_cast<uint64_t>(ha) << 32));
      f.k[b] = static_cast<K>(lb | (static_cast<uint64_t>(hb) << 32));
    }
    if constexpr (PAIRS) word(f.ix[a], f.ix[b], 2);
    if constexpr (PAIRS && VALS) word(f.v[a], f.v[b], 3);
  }
}

// The compare-exchange forms each kernel uses, per element kind: in the
// BLK-layout stages (Blk) and in the other stages and the per-thread network
// (Oth).  Block: the block sort; Merge: the merge passes, whose networks carry
// (key, rank) only (the payloads are gathered by rank afterwards); Piece: the
// segmented worker's merge pieces, which carry the payloads through the
// network.  The block sorts with payloads carry (key, position) only as well.
// Measured on GB300 (sweeps over the word choices).
template <typename K, bool PAIRS> struct CeForms;
template <> struct CeForms<uint32_t, false> {
  static constexpr int kBlockBlk = kFmaKeys, kBlockOth = 0;
  static constexpr int kMergeBlk = kFmaKeys, kMergeOth = 0;
  static constexpr int kPieceBlk = kMergeBlk, kPieceOth = kMergeOth;
};
template <> struct CeForms<uint32_t, true> {
  static constexpr int kBlockBlk = 0, kBlockOth = 0;
  static constexpr int kMergeBlk = kFmaWord(2), kMergeOth = 0;
  static constexpr int kPieceBlk = kFmaWord(3), kPieceOth = kFmaWord(3);
};
template <> struct CeForms<uint64_t, false> {
  static constexpr int kBlockBlk = kFmaWord(0) | kFmaWord(1), kBlockOth = 0;
  static constexpr int kMergeBlk = kFmaWord(0) | kFmaWord(1), kMergeOth = kFmaWord(0) | kFmaWord(1);
  static constexpr int kPieceBlk = 0, kPieceOth = 0;
};
template <> struct CeForms<uint64_t, true> {
  static constexpr int kBlockBlk = 0, kBlockOth = 0;
  static constexpr int kMergeBlk = kFmaWord(1) | kFmaWord(2), kMergeOth = 0;
  static constexpr int kPieceBlk = 0, kPieceOth = 0;
};

// Batcher's odd-even merge sort network on N inputs (Knuth vol. 3, Sec.
// 5.3.4, Algorithm M), listed as comparator pairs at compile time.
template <int N>
struct OemNetwork {
  int n;
  unsigned char a[N * 8], b[N * 8];
  constexpr OemNetwork() : n(0), a{}, b{} {
    for (int p = 1; p < N; p <<= 1)
      for (int kk = p; kk >= 1; kk >>= 1)
        for (int j = kk % p; j + kk < N; j += 2 * kk)
          for (int i = 0; i < kk; ++i)
            if (i + j + kk < N && (i + j) / (2 * p) == (i + j + kk) / (2 * p)) {
              a[n] = static_cast<unsigned char>(i + j);
              b[n] = static_cast<unsigned char>(i + j + kk);
              ++n;
            }
  }
};

// The "BATCHERS-ODD-EVEN-MERGESORT(R)" register network of Algorithms 1 and
// 2: sorts one thread's E registers, direction chosen per thread.
template <int FMA = 0, typename K, bool PAIRS, int E, bool VALS>
__device__ __forceinline__ void thread_sort(Frag<K, PAIRS, E, VALS>& f, bool desc) {
  constexpr OemNetwork<E> net{};
#pragma unroll
  for (int c = 0; c < net.n; ++c) ce(f, net.a[c], net.b[c], desc, FMA);
}

// ---------------------------------------------------------------- layouts
// Three register layouts of a CTA tile X[0, 2^t) with E = 2^r registers per
// thread, NT = 2^(t-r) threads, lane = tid & 31, warp = tid >> 5:
//   BLK  register window k bits [0, r)     k = tid*E + e
//   MID  register window k bits [r, 2r)    r = 5: k = warp<<10 | e<<5 | lane
//                                          r = 4: k = lane[0:4] | e<<4 |
//                                                 warp[0]<<8 | lane[4]<<9 |
//                                                 warp[1:]<<10
//   STR  register window k bits [t-r, t)   k = e*NT + tid
// For t <= 3r the windows cover every bit, so every stage of a bitonic
// network is an in-register compare-exchange in one of them.  Layouts change
// through shared memory padded with one word per 32 (word k lives at
// k + (k >> 5)).  A warp's 32 accesses then always hit 32 distinct banks:
//   STR, MID(r=5): lanes are k bits [0,5)        -> consecutive words
//   MID(r=4)     : lanes are k bits {0..3, 9}    -> banks l[0:4] + 16*l[4]
//   BLK          : lanes are k bits [r, r+5)     -> banks (l*E + l*E/32) mod 32
// which is the paper's row-per-thread / skewed-matrix principle (Sec. 2.1,
// Sec. 3.3 "implicit matrix transposition").  Every address is a per-thread
// base plus a compile-time offset, so layout changes cost no arithmetic.
enum { kBLK = 0, kMID = 1, kSTR = 2 };

template <int E, int NT>
struct Geo {
  static constexpr int r = ilog2(E);
  static constexpr int t = ilog2(E * NT);
  static constexpr uint32_t T = E * NT;
  static constexpr uint32_t kPlane = padded_words(T);
  static_assert(r == 4 || r == 5, "E must be 16 or 32");
  static_assert(t >= 10 && t <= 3 * r, "tile size outside what three layouts cover");

  template <int L>
  static constexpr int win() { return L == kBLK ? 0 : (L == kMID ? r : t - r); }

  // per-thread base of layout L; MIRROR: the base of the element whose index
  // has every bit below the register window flipped (lanes / threads mirrored)
  template <int L, bool MIRROR>
  __device__ static __forceinline__ uint32_t base(uint32_t tid) {
    if constexpr (L == kBLK) {
      static_assert(!MIRROR, "BLK is never read mirrored");
      const uint32_t k0 = tid * E;
      return k0 + (k0 >> 5);
    } else if constexpr (L == kSTR) {
      const uint32_t tt = MIRROR ? (tid ^ (NT - 1)) : tid;
      return tt + (tt >> 5);
    } else {
      const uint32_t w = tid >> 5, l = tid & 31;
      if constexpr (r == 5) {
        return w * 1056u + (MIRROR ? (l ^ 31u) : l);
      } else {
        const uint32_t lo = MIRROR ? ((l & 15u) ^ 15u) : (l & 15u);
        return lo + 264u * (w & 1u) + 528u * (l >> 4) + 1056u * (w >> 1);
      }
    }
  }
  template <int L>
  __host__ __device__ static constexpr uint32_t off(int e) {
    return L == kBLK ? static_cast<uint32_t>(e)
         : L == kSTR ? static_cast<uint32_t>(e) * (NT + NT / 32)
         : (r == 5 ? 33u * e : 16u * e + (e >> 1));
  }
};

// Layout change FROM -> TO through shared memory.  FLIPJ > 0 reverses the
// upper half of every 2^FLIPJ block while reading (element k of an upper half
// is fetched from k ^ (2^(FLIPJ-1) - 1)), turning two ascending halves into
// one bitonic sequence -- so every compare-exchange of the sort is ascending.
// Requires bit FLIPJ-1 to lie in TO's register window.
template <int FROM, int TO, int FLIPJ, int NT, typename K, bool PAIRS, int E, bool VALS>
__device__ __forceinline__ void relayout(Frag<K, PAIRS, E, VALS>& f, uint32_t* sm) {
  using G = Geo<E, NT>;
  const uint32_t tid = threadIdx.x;
  __syncthreads();
  {
    const uint32_t b = G::template base<FROM, false>(tid);
#pragma unroll
    for (int e = 0; e < E; ++e) f.put(sm, G::kPlane, e, b + G::template off<FROM>(e));
  }
  __syncthreads();
  const uint32_t b = G::template base<TO, false>(tid);
  if constexpr (FLIPJ == 0) {
#pragma unroll
    for (int e = 0; e < E; ++e) f.get(sm, G::kPlane, e, b + G::template off<TO>(e));
  } else {
    constexpr int q = FLIPJ - 1 - G::template win<TO>();  // register bit of k bit FLIPJ-1
    static_assert(q >= 0 && q < G::r, "flip bit outside the target window");
    const uint32_t bm = G::template base<TO, true>(tid);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (e & (1 << q))
        f.get(sm, G::kPlane, e, bm + G::template off<TO>(e ^ ((1 << q) - 1)));
      else
        f.get(sm, G::kPlane, e, b + G::template off<TO>(e));
    }
  }
}

// Ascending half-cleaner stages on k bits HI down to LO, all inside layout
// L's register window (FMA: the kFma* forms the compare-exchanges use).
template <int L, int HI, int LO, int NT, int FMA = 0, typename K, bool PAIRS, int E, bool VALS>
__device__ __forceinline__ void stages(Frag<K, PAIRS, E, VALS>& f) {
  using G = Geo<E, NT>;
#pragma unroll
  for (int b = HI; b >= LO; --b) {
    const int q = b - G::template win<L>();
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (!(e & (1 << q))) ce(f, e, e | (1 << q), false, FMA);
  }
}

// Bitonic merge of the bitonic sequence of length E*NT held in STR layout;
// ascending result in BLK layout.  Stages on bits t-1 .. 0 in STR, MID, BLK.
// Both layout changes reuse one buffer (a second buffer would save two
// barriers but halves the CTAs per SM, which was measured slower).
// FMA_BLK / FMA_OTH: the compare-exchange forms of the BLK stages / of the
// others (Frag::one must be set when either is non-zero).
template <int NT, int FMA_BLK = 0, int FMA_OTH = 0, typename K, bool PAIRS, int E, bool VALS>
__device__ __forceinline__ void bitonic_merge_str(Frag<K, PAIRS, E, VALS>& f, uint32_t* sm) {
  using G = Geo<E, NT>;
  constexpr int r = G::r, t = G::t;
  stages<kSTR, t - 1, t - r, NT, FMA_OTH>(f);
  if constexpr (t - r - 1 >= r) {
    relayout<kSTR, kMID, 0, NT>(f, sm);
    stages<kMID, t - r - 1, r, NT, FMA_OTH>(f);
    relayout<kMID, kBLK, 0, NT>(f, sm);
  } else {
    relayout<kSTR, kBLK, 0, NT>(f, sm);
  }
  stages<kBLK, r - 1, 0, NT, FMA_BLK>(f);
}

// Lane exchange of a compare-exchange whose two elements sit in lanes
// l and l ^ m of one warp: this lane's register a meets the partner lane's
// register b; the lower lane keeps the smaller element, the upper the larger.
// (key, tie-break index) order for pairs; the payload follows.
template <typename K, bool PAIRS, int E, bool VALS>
struct LaneVal {
  K k;
  uint32_t ix, v;
};
template <typename K, bool PAIRS, int E, bool VALS>
__device__ __forceinline__ LaneVal<K, PAIRS, E, VALS> lane_fetch(const Frag<K, PAIRS, E, VALS>& f,
                                                                 int b, uint32_t m) {
  LaneVal<K, PAIRS, E, VALS> y;
  y.k = __shfl_xor_sync(0xFFFFFFFFu, f.k[b], m);
  if constexpr (PAIRS) y.ix = __shfl_xor_sync(0xFFFFFFFFu, f.ix[b], m);
  if constexpr (PAIRS && VALS) y.v = __shfl_xor_sync(0xFFFFFFFFu, f.v[b], m);
  return y;
}
template <typename K, bool PAIRS, int E, bool VALS>
__device__ __forceinline__ void lane_keep(Frag<K, PAIRS, E, VALS>& f, int a,
                                          const LaneVal<K, PAIRS, E, VALS>& y, bool upper) {
  if constexpr (!PAIRS) {
    const K x = f.k[a];
    f.k[a] = upper ? (x > y.k ? x : y.k) : (x < y.k ? x : y.k);
  } else {
    const bool y_after = after(y.k, y.ix, f.k[a], f.ix[a]);
    const bool take = upper ? y_after : !y_after;
    f.k[a] = take ? y.k : f.k[a];
    f.ix[a] = take ? y.ix : f.ix[a];
    if constexpr (VALS) f.v[a] = take ? y.v : f.v[a];
  }
}

// Levels J with J - r <= shuffle_levels<K, PAIRS>() take their lane stages
// (k bits J-1 .. r, the lane bits of BLK) as warp shuffles instead of a BLK ->
// MID -> BLK round trip through shared memory: J - r shuffles of each word per
// element and no barrier, against two shared stores and two shared loads of
// each word and four barriers.  Measured on GB300 (block sort at 2^28): 32-bit
// keys gain up to four shuffle levels (1.84 -> 1.76 ms), elements of more than
// one word up to two (u64 keys 4.27 -> 4.19 ms, u64 + u32 payload 11.03 ->
// 10.69 ms; more levels were slower).
template <typename K, bool PAIRS>
__host__ __device__ constexpr int shuffle_levels() {
  return (!PAIRS && sizeof(K) == 4) ? 4 : 2;
}

// One level J of the bitonic sort in BLK layout with its lane stages done by
// shuffles.  The flip stage pairs element k with k ^ (2^J - 1): register e of
// lane l meets register E-1-e of lane l ^ (2^(J-r) - 1); the lower lane (k bit
// J-1 clear) keeps the minimum.  Then half-cleaners on lane bits, then the
// register stages r-1 .. 0.
template <int J, int NT, int FMA_BLK, int FMA_OTH, typename K, bool PAIRS, int E, bool VALS>
__device__ __forceinline__ void sort_level_shuffle(Frag<K, PAIRS, E, VALS>& f) {
  constexpr int r = ilog2(E);
  static_assert(J > r && J - r <= 5, "lane stages only");
  const uint32_t lane = threadIdx.x & 31u;
  {
    constexpr uint32_t m = (1u << (J - r)) - 1u;
    const bool upper = ((lane >> (J - 1 - r)) & 1u) != 0;
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {
      const LaneVal<K, PAIRS, E, VALS> y1 = lane_fetch(f, E - 1 - e, m);  // meets my e
      const LaneVal<K, PAIRS, E, VALS> y2 = lane_fetch(f, e, m);          // meets my E-1-e
      lane_keep(f, e, y1, upper);
      lane_keep(f, E - 1 - e, y2, upper);
    }
  }
#pragma unroll
  for (int b = J - 2; b >= r; --b) {
    const uint32_t m = 1u << (b - r);
    const bool upper = (lane & m) != 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const LaneVal<K, PAIRS, E, VALS> y = lane_fetch(f, e, m);
      lane_keep(f, e, y, upper);
    }
  }
  stages<kBLK, r - 1, 0, NT, FMA_BLK>(f);
}

// One level J of the bitonic sort (r < J <= t): the tile's blocks of 2^(J-1)
// are ascending; merge pairs of them into ascending blocks of 2^J.  Enters and
// leaves in BLK layout.  Low levels use lane shuffles (above).  A level whose
// top bit lies in the MID window [r, 2r) needs two layout changes (BLK -> MID
// -> BLK); only a level whose top bit lies above it goes through STR (three).
template <int J, int NT, int FMA_BLK, int FMA_OTH, typename K, bool PAIRS, int E, bool VALS>
__device__ __forceinline__ void sort_level(Frag<K, PAIRS, E, VALS>& f, uint32_t* sm) {
  using G = Geo<E, NT>;
  constexpr int r = G::r, t = G::t, top = J - 1;
  if constexpr (J - r <= shuffle_levels<K, PAIRS>()) {
    sort_level_shuffle<J, NT, FMA_BLK, FMA_OTH>(f);
    return;
  } else if constexpr (top >= 2 * r) {
    relayout<kBLK, kSTR, J, NT>(f, sm);
    stages<kSTR, top, t - r, NT, FMA_OTH>(f);
    if constexpr (t - r - 1 >= r) {
      relayout<kSTR, kMID, 0, NT>(f, sm);
      stages<kMID, t - r - 1, r, NT, FMA_OTH>(f);
      relayout<kMID, kBLK, 0, NT>(f, sm);
    } else {
      relayout<kSTR, kBLK, 0, NT>(f, sm);
    }
  } else {
    relayout<kBLK, kMID, J, NT>(f, sm);
    stages<kMID, top, r, NT, FMA_OTH>(f);
    relayout<kMID, kBLK, 0, NT>(f, sm);
  }
  stages<kBLK, r - 1, 0, NT, FMA_BLK>(f);
}

template <int J, int NT, int FMA_BLK, int FMA_OTH, typename K, bool PAIRS, int E, bool VALS,
          bool DONE = (J > ilog2(E * NT))>
struct SortLevels {
  __device__ static __forceinline__ void run(Frag<K, PAIRS, E, VALS>& f, uint32_t* sm) {
    sort_level<J, NT, FMA_BLK, FMA_OTH>(f, sm);
    SortLevels<J + 1, NT, FMA_BLK, FMA_OTH, K, PAIRS, E, VALS>::run(f, sm);
  }
};
template <int J, int NT, int FMA_BLK, int FMA_OTH, typename K, bool PAIRS, int E, bool VALS>
struct SortLevels<J, NT, FMA_BLK, FMA_OTH, K, PAIRS, E, VALS, true> {
  __device__ static __forceinline__ void run(Frag<K, PAIRS, E, VALS>&, uint32_t*) {}
};

// Sort of the whole CTA tile: each thread's registers with Batcher's network
// (levels 1..r), then levels r+1..t; ascending result in BLK layout.
// FMA_BLK / FMA_OTH: the compare-exchange forms of the BLK stages / of the
// per-thread network and the other stages (Frag::one must be set when either
// is non-zero).
template <int NT, int FMA_BLK = 0, int FMA_OTH = 0, typename K, bool PAIRS, int E, bool VALS>
__device__ __forceinline__ void block_sort_tile(Frag<K, PAIRS, E, VALS>& f, uint32_t* sm) {
  thread_sort<FMA_OTH>(f, false);
  SortLevels<ilog2(E) + 1, NT, FMA_BLK, FMA_OTH, K, PAIRS, E, VALS>::run(f, sm);
}

}  // namespace bcf
