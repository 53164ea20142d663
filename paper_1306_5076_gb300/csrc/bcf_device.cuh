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

// Register fragment: E elements per thread.  PAIRS carries the u32 payload
// and a tie-break index (the element's rank in the stable input order),
// because bitonic networks are not stable on their own.
template <typename K, bool PAIRS, int E>
struct Frag {
  static constexpr int KW = sizeof(K) / 4;           // 32-bit words per key
  static constexpr int W = KW + (PAIRS ? 2 : 0);     // 32-bit planes per element
  K k[E];
  uint32_t ix[PAIRS ? E : 1];
  uint32_t v[PAIRS ? E : 1];
  uint32_t one;  // the multiplier of the FMA-pipe maximum (see ce()); set by kernels that use it

  __device__ __forceinline__ void put(uint32_t* sm, uint32_t plane, int e, uint32_t a) const {
    sm[a] = static_cast<uint32_t>(k[e]);
    if constexpr (KW == 2) sm[plane + a] = static_cast<uint32_t>(static_cast<uint64_t>(k[e]) >> 32);
    if constexpr (PAIRS) {
      sm[KW * plane + a] = ix[e];
      sm[(KW + 1) * plane + a] = v[e];
    }
  }
  __device__ __forceinline__ void get(const uint32_t* sm, uint32_t plane, int e, uint32_t a) {
    if constexpr (KW == 2)
      k[e] = static_cast<K>(sm[a]) | (static_cast<K>(sm[plane + a]) << 32);
    else
      k[e] = static_cast<K>(sm[a]);
    if constexpr (PAIRS) {
      ix[e] = sm[KW * plane + a];
      v[e] = sm[(KW + 1) * plane + a];
    }
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
    return kx > ky || (kx == ky && ix > iy);
  }
}

// A 1 that the compiler cannot fold away (it could be written from the host),
// read once per thread into Frag::one.
static __device__ uint32_t g_unit_multiplier = 1;

// Work moved from the ALU pipe, which the sorting networks keep saturated, to
// the FMA pipe (integer multiply-adds with a multiplier of Frag::one), in the
// compare-exchanges of the stages that ask for it (measured: the BLK-layout
// stages).  Both forms are exact in modular arithmetic.
//   kFmaKeys  (32-bit keys, no payloads): the maximum is x * 1 + y - min(x, y)
//             instead of a second min/max;
//   kFmaPairs (32-bit keys with payloads): each of the three words is swapped
//             as x + s * (y - x), y' = x + y - x' with s = 0 or 1, instead of
//             two selects;
//   kFmaKeys64 (64-bit keys, no payloads): the same swap of the two halves
//             after one 64-bit comparison, instead of four selects.
enum : int { kFmaKeys = 1, kFmaPairs = 2, kFmaKeys64 = 4 };

// Compare-exchange registers a < b: ascending puts the smaller element in a.
template <typename K, bool PAIRS, int E>
__device__ __forceinline__ void ce(Frag<K, PAIRS, E>& f, int a, int b, bool desc, int fma = 0) {
  if (!PAIRS && sizeof(K) == 4 && (fma & kFmaKeys)) {
    const uint32_t x = static_cast<uint32_t>(f.k[a]), y = static_cast<uint32_t>(f.k[b]);
    const uint32_t lo = x < y ? x : y;
    uint32_t hi;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(hi) : "r"(x), "r"(f.one), "r"(y));
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(hi) : "r"(lo), "r"(0u - f.one), "r"(hi));
    f.k[a] = static_cast<K>(desc ? hi : lo);
    f.k[b] = static_cast<K>(desc ? lo : hi);
  } else if (!PAIRS && sizeof(K) == 8 && (fma & kFmaKeys64)) {
    const uint64_t x = static_cast<uint64_t>(f.k[a]), y = static_cast<uint64_t>(f.k[b]);
    const bool sw = (x > y) != desc;
    const uint32_t s = sw ? f.one : 0u, one = f.one, neg = 0u - f.one;
    uint32_t xw[2] = {static_cast<uint32_t>(x), static_cast<uint32_t>(x >> 32)};
    uint32_t yw[2] = {static_cast<uint32_t>(y), static_cast<uint32_t>(y >> 32)};
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      uint32_t d, nx, t, ny;
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(xw[w]), "r"(neg), "r"(yw[w]));
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(nx) : "r"(s), "r"(d), "r"(xw[w]));
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(t) : "r"(xw[w]), "r"(one), "r"(yw[w]));
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(ny) : "r"(nx), "r"(neg), "r"(t));
      xw[w] = nx;
      yw[w] = ny;
    }
    f.k[a] = static_cast<K>(xw[0] | (static_cast<uint64_t>(xw[1]) << 32));
    f.k[b] = static_cast<K>(yw[0] | (static_cast<uint64_t>(yw[1]) << 32));
  } else if constexpr (!PAIRS) {
    const K x = f.k[a], y = f.k[b];
    const K lo = x < y ? x : y, hi = x < y ? y : x;
    f.k[a] = desc ? hi : lo;
    f.k[b] = desc ? lo : hi;
  } else if (sizeof(K) == 4 && (fma & kFmaPairs)) {
    const bool sw = after(f.k[a], f.ix[a], f.k[b], f.ix[b]) != desc;
    const uint32_t s = sw ? f.one : 0u, one = f.one, neg = 0u - f.one;
    const auto swap_word = [&](uint32_t& xr, uint32_t& yr) {
      const uint32_t x = xr, y = yr;
      uint32_t d, nx, t, ny;
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(neg), "r"(y));    // y - x
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(nx) : "r"(s), "r"(d), "r"(x));     // x + s(y - x)
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(t) : "r"(x), "r"(one), "r"(y));    // x + y
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(ny) : "r"(nx), "r"(neg), "r"(t));  // x + y - x'
      xr = nx;
      yr = ny;
    };
    uint32_t ka = static_cast<uint32_t>(f.k[a]), kb = static_cast<uint32_t>(f.k[b]);
    swap_word(ka, kb);
    f.k[a] = static_cast<K>(ka);
    f.k[b] = static_cast<K>(kb);
    swap_word(f.ix[a], f.ix[b]);
    swap_word(f.v[a], f.v[b]);
  } else {
    const bool sw = after(f.k[a], f.ix[a], f.k[b], f.ix[b]) != desc;
    const K ka = f.k[a], kb = f.k[b];
    const uint32_t ia = f.ix[a], ib = f.ix[b], va = f.v[a], vb = f.v[b];
    f.k[a] = sw ? kb : ka;
    f.k[b] = sw ? ka : kb;
    f.ix[a] = sw ? ib : ia;
    f.ix[b] = sw ? ia : ib;
    f.v[a] = sw ? vb : va;
    f.v[b] = sw ? va : vb;
  }
}

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
template <typename K, bool PAIRS, int E>
__device__ __forceinline__ void thread_sort(Frag<K, PAIRS, E>& f, bool desc) {
  constexpr OemNetwork<E> net{};
#pragma unroll
  for (int c = 0; c < net.n; ++c) ce(f, net.a[c], net.b[c], desc);
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
template <int FROM, int TO, int FLIPJ, int NT, typename K, bool PAIRS, int E>
__device__ __forceinline__ void relayout(Frag<K, PAIRS, E>& f, uint32_t* sm) {
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
template <int L, int HI, int LO, int NT, int FMA = 0, typename K, bool PAIRS, int E>
__device__ __forceinline__ void stages(Frag<K, PAIRS, E>& f) {
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
// FMA_BLK: the kFma* forms of the BLK stages (Frag::one must be set).
template <int NT, int FMA_BLK = 0, typename K, bool PAIRS, int E>
__device__ __forceinline__ void bitonic_merge_str(Frag<K, PAIRS, E>& f, uint32_t* sm) {
  using G = Geo<E, NT>;
  constexpr int r = G::r, t = G::t;
  stages<kSTR, t - 1, t - r, NT>(f);
  if constexpr (t - r - 1 >= r) {
    relayout<kSTR, kMID, 0, NT>(f, sm);
    stages<kMID, t - r - 1, r, NT>(f);
    relayout<kMID, kBLK, 0, NT>(f, sm);
  } else {
    relayout<kSTR, kBLK, 0, NT>(f, sm);
  }
  stages<kBLK, r - 1, 0, NT, FMA_BLK>(f);
}

// One level J of the bitonic sort (r < J <= t): the tile's blocks of 2^(J-1)
// are ascending; merge pairs of them into ascending blocks of 2^J.  Enters and
// leaves in BLK layout.
template <int J, int NT, int FMA_BLK, typename K, bool PAIRS, int E>
__device__ __forceinline__ void sort_level(Frag<K, PAIRS, E>& f, uint32_t* sm) {
  using G = Geo<E, NT>;
  constexpr int r = G::r, t = G::t, top = J - 1;
  if constexpr (top >= t - r) {
    relayout<kBLK, kSTR, J, NT>(f, sm);
    stages<kSTR, top, t - r, NT>(f);
    if constexpr (t - r - 1 >= r) {
      relayout<kSTR, kMID, 0, NT>(f, sm);
      stages<kMID, t - r - 1, r, NT>(f);
      relayout<kMID, kBLK, 0, NT>(f, sm);
    } else {
      relayout<kSTR, kBLK, 0, NT>(f, sm);
    }
  } else {
    relayout<kBLK, kMID, J, NT>(f, sm);
    stages<kMID, top, r, NT>(f);
    relayout<kMID, kBLK, 0, NT>(f, sm);
  }
  stages<kBLK, r - 1, 0, NT, FMA_BLK>(f);
}

template <int J, int NT, int FMA_BLK, typename K, bool PAIRS, int E,
          bool DONE = (J > ilog2(E * NT))>
struct SortLevels {
  __device__ static __forceinline__ void run(Frag<K, PAIRS, E>& f, uint32_t* sm) {
    sort_level<J, NT, FMA_BLK>(f, sm);
    SortLevels<J + 1, NT, FMA_BLK, K, PAIRS, E>::run(f, sm);
  }
};
template <int J, int NT, int FMA_BLK, typename K, bool PAIRS, int E>
struct SortLevels<J, NT, FMA_BLK, K, PAIRS, E, true> {
  __device__ static __forceinline__ void run(Frag<K, PAIRS, E>&, uint32_t*) {}
};

// Sort of the whole CTA tile: each thread's registers with Batcher's network
// (levels 1..r), then levels r+1..t; ascending result in BLK layout.
// FMA_BLK: the kFma* forms of the BLK stages (Frag::one must be set).
template <int NT, int FMA_BLK = 0, typename K, bool PAIRS, int E>
__device__ __forceinline__ void block_sort_tile(Frag<K, PAIRS, E>& f, uint32_t* sm) {
  thread_sort(f, false);
  SortLevels<ilog2(E) + 1, NT, FMA_BLK, K, PAIRS, E>::run(f, sm);
}

}  // namespace bcf
