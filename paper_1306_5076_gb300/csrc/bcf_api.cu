// bcf_api.cu -- the C ABI declared in include/bcfsort.h: argument checks,
// workspace layout, pass planning and kernel sequencing.
//
// A sort of n keys is the paper's BCFMergesort (Sec. 3; Lemma 2): one base-
// case pass (block sort of T-key tiles) then ceil(log2(n / T)) merge passes,
// each one read and one write of the data.  Passes ping-pong between the
// caller's output buffer and the workspace so that the last pass lands in the
// output.  Keys are mapped to unsigned order when first read and mapped back
// when last written, so intermediate passes compare plain unsigned integers.
#include <cuda_runtime.h>

#include <dlfcn.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bcf_internal.h"
#include "bcfsort.h"

namespace bcf {

__device__ uint32_t g_error_word;  // set by bounded waits that ran out

// Run-time settings read by the launch wrappers (bcf_internal.h).
static std::atomic<uint64_t> g_wait_limit_ns{kDefaultWaitLimitNs};
static std::atomic<uint32_t> g_smem_floor{0};
static std::atomic<bool> g_profiling{false};
uint64_t wait_limit_ns() { return g_wait_limit_ns.load(std::memory_order_relaxed); }
uint32_t smem_floor_bytes() { return g_smem_floor.load(std::memory_order_relaxed); }
bool chained_launches() { return !g_profiling.load(std::memory_order_relaxed); }

namespace {


bool dtype_ok(int kt) { return kt >= BCF_U32 && kt <= BCF_I16; }
bool is16(int kt) { return kt == BCF_U16 || kt == BCF_I16; }
int key_bytes_of(bcf_dtype kt) {
  if (is16(kt)) return 2;
  return (kt == BCF_U64 || kt == BCF_I64 || kt == BCF_F64) ? 8 : 4;
}
// 16-bit keys go through the 32-bit sort: zero- (u16) or sign-extended (i16).
bcf_dtype wide_of(bcf_dtype kt) { return kt == BCF_U16 ? BCF_U32 : BCF_I32; }

// The key map of the device code: bit 0 totalOrder (f32 / f64), bit 2
// two's-complement (i32 / i64), bit 1 descending.
int mode_of(bcf_dtype kt, const bcf_opts* o) {
  int m = 0;
  if (kt == BCF_F32 || kt == BCF_F64) m |= 1;
  if (kt == BCF_I32 || kt == BCF_I64) m |= 4;
  if (o && o->descending) m |= 2;
  return m;
}

// ---------------------------------------------------------------- tuning
//
// (E, NT) per operation, key width, payload flag and size band come from a
// table: bcf_tuning_set() installs one; otherwise the first call reads the
// committed table "tuning/gb300.tsv" next to the package directory of this
// library (written by the project's autotuner, paper_1306_5076_gb300/autotune.py),
// and without a table the built-in defaults below apply.

struct Tuning {
  int block_cfg, merge_cfg;
};

struct TuneTable {
  std::mutex mu;
  bool loaded = false;
  std::vector<bcf_tuning_entry> rows;
};
TuneTable& tune_table() {
  static TuneTable t;
  return t;
}

bool entry_ok(const bcf_tuning_entry& e) {
  const bool pairs = e.has_vals != 0;
  if (e.key_bytes != 4 && e.key_bytes != 8) return false;
  if (e.n_max <= e.n_min) return false;
  if (e.op == BCF_OP_SORT || e.op == BCF_OP_MERGE) {
    if (!block_cfg_supported(e.key_bytes, pairs, e.block_cfg)) return false;
    if (!merge_cfg_supported(e.key_bytes, pairs, e.merge_cfg)) return false;
    return kMergeCfgs[e.merge_cfg].tile() <= 2 * kBlockCfgs[e.block_cfg].tile();
  }
  if (e.op == BCF_OP_SEGMENTED) {
    // merge_cfg -1: the worker merges; else the merge passes of multi-tile
    // segments are launches of that merge configuration, whose tile must
    // divide the segmented sort's tile
    if (!seg_cfg_supported(e.key_bytes, pairs, e.seg_cfg)) return false;
    if (e.merge_cfg == -1) return true;
    return merge_cfg_supported(e.key_bytes, pairs, e.merge_cfg) &&
           kMergeCfgs[e.merge_cfg].tile() <= kSegCfgs[e.seg_cfg].tile();
  }
  return false;
}

// Table file: '#' comments; rows "op key_bytes has_vals n_min n_max block merge seg".
void load_table_file(std::vector<bcf_tuning_entry>& rows) {
  Dl_info info{};
  if (!dladdr(reinterpret_cast<void*>(&load_table_file), &info) || !info.dli_fname) return;
  std::string path(info.dli_fname);
  const size_t slash = path.rfind('/');
  if (slash == std::string::npos) return;
  path = path.substr(0, slash) + "/../tuning/gb300.tsv";  // <pkg>/_build/lib -> <pkg>/tuning
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    bcf_tuning_entry e{};
    unsigned long long lo = 0, hi = 0;
    if (std::sscanf(line, "%d %d %d %llu %llu %d %d %d", &e.op, &e.key_bytes, &e.has_vals, &lo,
                    &hi, &e.block_cfg, &e.merge_cfg, &e.seg_cfg) == 8) {
      e.n_min = lo;
      e.n_max = hi;
      if (entry_ok(e)) rows.push_back(e);
    }
  }
  std::fclose(f);
}

const bcf_tuning_entry* find_entry(int op, int kb, bool pairs, uint64_t n) {
  TuneTable& t = tune_table();
  std::lock_guard<std::mutex> lk(t.mu);
  if (!t.loaded) {
    load_table_file(t.rows);
    t.loaded = true;
  }
  for (const auto& e : t.rows)
    if (e.op == op && e.key_bytes == kb && (e.has_vals != 0) == pairs && n >= e.n_min &&
        n < e.n_max)
      return &e;
  return nullptr;
}

// Built-in defaults (measured on GB300 at 2^28 keys): u32 keys-only use
// 8192-key block tiles (32 x 256) and 2048-key merge tiles (16 x 128); pairs
// and 64-bit keys use 4096-key block tiles (16 x 256).
Tuning tuning_for(int op, int kb, bool pairs, uint64_t n) {
  if (const bcf_tuning_entry* e = find_entry(op, kb, pairs, n)) return {e->block_cfg, e->merge_cfg};
  if (kb == 4 && !pairs) return {1, 3};
  return {0, 3};
}

struct Plan {
  Tuning tune;
  uint32_t T, Tm, passes;
};

Plan make_plan(uint64_t n, int kb, bool pairs, int op = BCF_OP_SORT) {
  Plan p;
  p.tune = tuning_for(op, kb, pairs, n);
  p.T = kBlockCfgs[p.tune.block_cfg].tile();
  p.Tm = kMergeCfgs[p.tune.merge_cfg].tile();
  p.passes = 0;
  uint64_t runs = (n + p.T - 1) / p.T;
  while (runs > 1) {
    runs = (runs + 1) / 2;
    ++p.passes;
  }
  return p;
}

// Segmented sort workspace: counters, per-segment state, the work queue and
// one copy of the keys (+ values).  The queue bound holds for any segment
// sizes: a segment touches at most size/T + 2 tiles, and each of its passes
// has one item per tile.
struct SegLayout {
  size_t ctl, items, tiny, tbase, splits, queue, order, pend, count_ge, pitems, chunks, pnext,
      samp0, samp1, keys, vals, total;
  uint64_t capacity;
};

SegLayout seg_layout(uint64_t n, uint64_t nseg, int kb, bool pairs) {
  SegLayout w;
  const uint64_t tiles = n / kMinSegTile + 2 * nseg + 2;
  uint64_t passes = 1;
  while ((1ull << passes) < tiles) ++passes;
  w.capacity = tiles * (1 + passes) + nseg / 4 + 2;  // tiny groups: >= 4 per item
  w.ctl = kAlign;
  w.items = align_up(w.ctl + seg_ctl_bytes(), kAlign);
  w.tiny = align_up(w.items + nseg * 4, kAlign);
  w.tbase = align_up(w.tiny + nseg * 4, kAlign);
  w.splits = align_up(w.tbase + nseg * 8, kAlign);
  w.queue = align_up(w.splits + tiles * 8, kAlign);
  // merge passes outside the worker: the segment list, and one record per
  // merge tile (at most `tiles` of them; the splits above serve them too)
  w.order = align_up(w.queue + w.capacity * seg_work_bytes(), kAlign);
  w.pend = align_up(w.order + nseg * 4, kAlign);
  w.count_ge = align_up(w.pend + nseg * 8, kAlign);
  w.pitems = align_up(w.count_ge + (kSegMaxPasses + 2) * 4, kAlign);
  // samples of the output and of the keys copy for the launches' partitions
  const uint64_t nsamp = n / kRunSampleStride + 2;
  w.chunks = align_up(w.pitems + tiles * sizeof(SegItem), kAlign);
  w.pnext = align_up(w.chunks + (tiles / 32 + 2) * 4, kAlign);
  w.samp0 = align_up(w.pnext + (kSegMaxPasses + 2) * 8, kAlign);
  w.samp1 = align_up(w.samp0 + nsamp * kb, kAlign);
  w.keys = align_up(w.samp1 + nsamp * kb, kAlign);
  w.vals = align_up(w.keys + n * kb, kAlign);
  w.total = align_up(w.vals + (pairs ? n * 4 : 0), kAlign);
  return w;
}

// Segmented sort: the worker's configuration and who merges (merge_cfg -1:
// the worker; else launches of that merge configuration).  Built-in default:
// 4096-key tiles (16 x 256), merges in the worker.
struct SegTuning {
  int seg_cfg, merge_cfg;
};
SegTuning seg_tuning_for(int kb, bool pairs, uint64_t n) {
  if (const bcf_tuning_entry* e = find_entry(BCF_OP_SEGMENTED, kb, pairs, n))
    return {e->seg_cfg, e->merge_cfg};
  return {0, -1};
}

// ---------------------------------------------------------------- device error word

uint32_t* error_word_ptr() {
  static std::mutex mu;
  static uint32_t* ptrs[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_error_word) != cudaSuccess) return nullptr;
    ptrs[dev] = static_cast<uint32_t*>(p);
  }
  return ptrs[dev];
}

// ---------------------------------------------------------------- profiling

struct Profiler {
  std::mutex mu;
  bool on = false;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
Profiler& prof() {
  static Profiler p;
  return p;
}

template <typename F>
cudaError_t timed(int kind, cudaStream_t s, F&& launch) {
  Profiler& P = prof();
  bool on;
  {
    std::lock_guard<std::mutex> lk(P.mu);
    on = P.on;
  }
  if (!on) return launch();
  cudaEvent_t a, b;
  {
    std::lock_guard<std::mutex> lk(P.mu);
    a = P.get();
    b = P.get();
  }
  cudaEventRecord(a, s);
  const cudaError_t err = launch();
  cudaEventRecord(b, s);
  std::lock_guard<std::mutex> lk(P.mu);
  P.pending.push_back({kind, a, b});
  return err;
}

// ---------------------------------------------------------------- argument checks

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct Span {
  const void* p;
  size_t bytes;
};
bool overlap(Span a, Span b) {
  if (!a.p || !b.p || a.bytes == 0 || b.bytes == 0) return false;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(a.p), b0 = reinterpret_cast<uintptr_t>(b.p);
  return a0 < b0 + b.bytes && b0 < a0 + a.bytes;
}
// out may equal in exactly; any other overlap among the spans is an error
bool bad_overlap(Span out, Span in) { return out.p != in.p && overlap(out, in); }

bcf_status check_common(void* ko, uint32_t* vo, const void* ki, const uint32_t* vi, uint64_t n,
                        int kt, bool pairs) {
  if (!dtype_ok(kt)) return BCF_EINVAL;
  if (n == 0) return BCF_OK;
  if (!ko || !ki) return BCF_EINVAL;
  if (pairs && (!vo || !vi)) return BCF_EINVAL;
  if (!aligned16(ko) || !aligned16(ki)) return BCF_EINVAL;
  if (pairs && (!aligned16(vo) || !aligned16(vi))) return BCF_EINVAL;
  const size_t kb = key_bytes_of(static_cast<bcf_dtype>(kt));
  const Span sko{ko, n * kb}, ski{ki, n * kb};
  if (bad_overlap(sko, ski)) return BCF_EINVAL;
  if (pairs) {
    const Span svo{vo, n * 4}, svi{vi, n * 4};
    if (bad_overlap(svo, svi) || overlap(sko, svo) || overlap(sko, svi) || overlap(ski, svo))
      return BCF_EINVAL;
  }
  return BCF_OK;
}

bcf_status check_ws(void* ws, size_t ws_bytes, size_t need, void* ko, uint32_t* vo,
                    const void* ki, const uint32_t* vi, uint64_t n, int kb) {
  if (ws_bytes < need || (need > 0 && !ws)) return BCF_ENOMEM;
  if (need == 0) return BCF_OK;
  if (!aligned16(ws)) return BCF_EINVAL;
  const Span sw{ws, need};
  if (overlap(sw, {ko, n * kb}) || overlap(sw, {ki, n * kb}) || overlap(sw, {vo, vo ? n * 4 : 0}) ||
      overlap(sw, {vi, vi ? n * 4 : 0}))
    return BCF_EINVAL;
  return BCF_OK;
}

bcf_status from_cuda(cudaError_t e) { return e == cudaSuccess ? BCF_OK : BCF_ECUDA; }

// ---------------------------------------------------------------- sort


// Input that arrives in pieces (bcf_sort_*_host): `before_tiles(t0, t1, s)`
// is called before the block sort of tiles [t0, t1) is launched on `s` and
// makes `s` wait until those tiles' input has landed.
struct ChunkedInput {
  uint64_t chunk_tiles;
  bcf_status (*before_tiles)(void* ctx, uint64_t t0, uint64_t t1, cudaStream_t s);
  void* ctx;
};

bcf_status run_sort(void* ko, uint32_t* vo, const void* ki, const uint32_t* vi, uint64_t n,
                    bcf_dtype kt, const bcf_opts* o, void* ws, size_t ws_bytes, cudaStream_t s,
                    bool pairs, const ChunkedInput* chunked = nullptr) {
  bcf_status st = check_common(ko, vo, ki, vi, n, kt, pairs);
  if (st != BCF_OK || n == 0) return st;
  const int kb = key_bytes_of(kt);
  const Plan plan = make_plan(n, kb, pairs);
  const WsLayout wl = ws_layout(n, 0, kb, pairs);
  const size_t need = plan.passes > 0 ? wl.total : 0;
  st = check_ws(ws, ws_bytes, need, ko, vo, ki, vi, n, kb);
  if (st != BCF_OK) return st;
  const int mode = mode_of(kt, o);
  uint32_t* err = error_word_ptr();
  if (!err) return BCF_ECUDA;

  char* wsb = static_cast<char*>(ws);
  void* kbuf[2] = {ko, plan.passes > 0 ? wsb + wl.keys : nullptr};
  uint32_t* vbuf[2] = {vo, (pairs && plan.passes > 0) ? reinterpret_cast<uint32_t*>(wsb + wl.vals)
                                                      : nullptr};
  const int m = static_cast<int>(plan.passes);
  // buffer written by pass i (0 = block sort): the output for i == m, and
  // alternating backwards from there
  auto buf = [m](int i) { return ((m - i) % 2 == 0) ? 0 : 1; };

  // sample arrays of the two buffers (the final output needs none)
  void* samp[2] = {plan.passes > 0 ? wsb + wl.samples0 : nullptr,
                   plan.passes > 0 ? wsb + wl.samples1 : nullptr};
  // the base case, in one launch or (input arriving in pieces) one launch per
  // chunk of whole tiles; a chunk's sample slots start at its first key / 256
  const uint64_t tiles = (n + plan.T - 1) / plan.T;
  const uint64_t step_tiles = chunked ? chunked->chunk_tiles : tiles;
  cudaError_t e = cudaSuccess;
  for (uint64_t t0 = 0; t0 < tiles; t0 += step_tiles) {
    const uint64_t t1 = t0 + step_tiles < tiles ? t0 + step_tiles : tiles;
    const uint64_t off = t0 * plan.T, len = (t1 * plan.T < n ? t1 * plan.T : n) - off;
    if (chunked && (st = chunked->before_tiles(chunked->ctx, t0, t1, s)) != BCF_OK) return st;
    void* sp = m == 0 ? nullptr : static_cast<char*>(samp[buf(0)]) + (off / kSampleStride) * kb;
    BlockSortArgs ba{static_cast<const char*>(ki) + off * kb, vi ? vi + off : nullptr,
                     static_cast<char*>(kbuf[buf(0)]) + off * kb,
                     vbuf[buf(0)] ? vbuf[buf(0)] + off : nullptr, len, mode, m == 0 ? mode : 0, sp};
    e = timed(0, s, [&] { return launch_block_sort(kb, pairs, plan.tune.block_cfg, ba, s); });
    if (e != cudaSuccess) return BCF_ECUDA;
  }
  uint64_t* splits = reinterpret_cast<uint64_t*>(wsb + wl.splits);
  const uint64_t items = (n + plan.Tm - 1) / plan.Tm;
  for (int i = 1; i <= m; ++i) {
    MergeArgs ma{};
    ma.kin = kbuf[buf(i - 1)];
    ma.vin = vbuf[buf(i - 1)];
    ma.kout = kbuf[buf(i)];
    ma.vout = vbuf[buf(i)];
    ma.n = n;
    ma.run = static_cast<uint64_t>(plan.T) << (i - 1);
    ma.run_log2 = static_cast<uint32_t>(ilog2_u64(plan.T)) + static_cast<uint32_t>(i - 1);
    ma.splits = splits;
    ma.mode_in = 0;
    ma.mode_out = i == m ? mode : 0;
    ma.err = err;
    ma.nitems = items;
    ma.samples_in = samp[buf(i - 1)];
    ma.samples_out = i == m ? nullptr : samp[buf(i)];
    e = timed(1, s, [&] { return launch_partition(kb, plan.tune.merge_cfg, ma, nullptr, s); });
    if (e != cudaSuccess) return BCF_ECUDA;
    e = timed(2, s, [&] { return launch_merge(kb, pairs, plan.tune.merge_cfg, ma, nullptr, s); });
    if (e != cudaSuccess) return BCF_ECUDA;
  }
  return BCF_OK;
}

// ---------------------------------------------------------------- merge runs

struct Run {
  uint64_t off, len;
};

bcf_status run_merge(void* ko, uint32_t* vo, const void* ki, const uint32_t* vi,
                     const uint64_t* offs, uint32_t k, bcf_dtype kt, const bcf_opts* o, void* ws,
                     size_t ws_bytes, cudaStream_t s) {
  const bool pairs = vo != nullptr || vi != nullptr;
  if (!offs || k == 0) return BCF_EINVAL;
  for (uint32_t r = 0; r < k; ++r)
    if (offs[r + 1] < offs[r]) return BCF_EINVAL;
  const uint64_t n = offs[k];  // arrays span [0, offs[k]); runs cover [offs[0], offs[k])
  bcf_status st = check_common(ko, vo, ki, vi, n, kt, pairs);
  if (st != BCF_OK) return st;
  if (offs[k] == offs[0]) return BCF_OK;
  const int kb = key_bytes_of(kt);
  const WsLayout wl = ws_layout(n, k, kb, pairs);
  st = check_ws(ws, ws_bytes, wl.total, ko, vo, ki, vi, n, kb);
  if (st != BCF_OK) return st;
  const int mode = mode_of(kt, o);
  uint32_t* err = error_word_ptr();
  if (!err) return BCF_ECUDA;
  const Plan plan = make_plan(n, kb, pairs, BCF_OP_MERGE);
  const uint64_t Tm = plan.Tm;
  const uint64_t lo = offs[0], span = offs[k] - offs[0];

  std::vector<Run> runs;
  runs.reserve(k);
  for (uint32_t r = 0; r < k; ++r) runs.push_back({offs[r], offs[r + 1] - offs[r]});
  int m = 0;
  for (size_t c = runs.size(); c > 1; c = (c + 1) / 2) ++m;

  char* wsb = static_cast<char*>(ws);
  void* wk = wsb + wl.keys;
  uint32_t* wv = pairs ? reinterpret_cast<uint32_t*>(wsb + wl.vals) : nullptr;
  const bool alias = ko == ki || (pairs && vo == vi);
  if (m == 0) {
    // a single run is already merged: copy it (identity key map both ways)
    if (ko != ki &&
        cudaMemcpyAsync(static_cast<char*>(ko) + lo * kb, static_cast<const char*>(ki) + lo * kb,
                        span * kb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return BCF_ECUDA;
    if (pairs && vo != vi &&
        cudaMemcpyAsync(vo + lo, vi + lo, span * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return BCF_ECUDA;
    return BCF_OK;
  }
  // pass i reads B[i-1] and writes B[i]; B[m] = output, alternating backwards.
  // With an aliased output and an odd pass count, pass 1 would write the
  // buffer it reads, so the input is first copied into the workspace.
  const void* src_k = ki;
  const uint32_t* src_v = vi;
  int src_mode = mode;
  if (alias && (m % 2 == 1)) {
    if (cudaMemcpyAsync(static_cast<char*>(wk) + lo * kb, static_cast<const char*>(ki) + lo * kb,
                        span * kb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return BCF_ECUDA;
    if (pairs && cudaMemcpyAsync(wv + lo, vi + lo, span * 4, cudaMemcpyDeviceToDevice, s) !=
                     cudaSuccess)
      return BCF_ECUDA;
    src_k = wk;
    src_v = wv;
  }
  uint64_t* splits = reinterpret_cast<uint64_t*>(wsb + wl.splits);
  // Samples (the keys at array positions that are multiples of
  // kRunSampleStride, in mapped order) narrow every merge-path search to a
  // window: pass i reads samp[i & 1], its merge kernel writes the next pass's
  // into samp[(i + 1) & 1], and pass 1's are taken from the input first.
  void* samp[2] = {wsb + wl.samples0, wsb + wl.samples1};
  if (launch_sample_span(kb, src_k, samp[1], src_mode, lo, offs[k], s) != cudaSuccess)
    return BCF_ECUDA;
  for (int i = 1; i <= m; ++i) {
    const bool to_out = ((m - i) % 2) == 0;
    void* dst_k = to_out ? ko : wk;
    uint32_t* dst_v = to_out ? vo : wv;
    // pair adjacent runs; an odd last run pairs with an empty one (a copy)
    std::vector<PairDesc> pairs_v;
    std::vector<Run> next;
    uint64_t piece = 0;
    for (size_t r = 0; r < runs.size(); r += 2) {
      const Run A = runs[r];
      const Run B = r + 1 < runs.size() ? runs[r + 1] : Run{A.off + A.len, 0};
      const uint64_t len = A.len + B.len;
      next.push_back({A.off, len});
      if (len == 0) continue;
      const uint64_t pieces = (A.off + len - 1) / Tm - A.off / Tm + 1;
      pairs_v.push_back({A.off, A.len, B.len, piece});
      piece += pieces;
    }
    for (size_t c = 0; c < pairs_v.size(); c += kMaxPairsPerLaunch) {
      PairList pl{};
      const size_t cnt = std::min<size_t>(kMaxPairsPerLaunch, pairs_v.size() - c);
      for (size_t q = 0; q < cnt; ++q) pl.p[q] = pairs_v[c + q];
      pl.npairs = static_cast<uint32_t>(cnt);
      const uint64_t end_piece = c + cnt < pairs_v.size() ? pairs_v[c + cnt].piece0 : piece;
      MergeArgs ma{};
      ma.kin = src_k;
      ma.vin = src_v;
      ma.kout = dst_k;
      ma.vout = dst_v;
      ma.n = n;
      ma.run = 0;
      ma.splits = splits;
      ma.mode_in = src_mode;
      ma.mode_out = i == m ? mode : 0;
      ma.err = err;
      ma.nitems = end_piece - pl.p[0].piece0;
      ma.samples_in = samp[i & 1];
      ma.samples_out = i == m ? nullptr : samp[(i + 1) & 1];
      cudaError_t e =
          timed(1, s, [&] { return launch_partition(kb, plan.tune.merge_cfg, ma, &pl, s); });
      if (e != cudaSuccess) return BCF_ECUDA;
      e = timed(2, s, [&] { return launch_merge(kb, pairs, plan.tune.merge_cfg, ma, &pl, s); });
      if (e != cudaSuccess) return BCF_ECUDA;
    }
    runs.swap(next);
    src_k = dst_k;
    src_v = dst_v;
    src_mode = 0;
  }
  return BCF_OK;
}

// ---------------------------------------------------------------- segmented

bcf_status run_segmented(void* ko, uint32_t* vo, const void* ki, const uint32_t* vi,
                         const uint64_t* off, uint64_t nseg, uint64_t n, bcf_dtype kt,
                         const bcf_opts* o, void* ws, size_t ws_bytes, cudaStream_t s,
                         bool skip_odd = false) {
  const bool pairs = vo != nullptr || vi != nullptr;
  if (pairs && (!vo || !vi)) return BCF_EINVAL;
  bcf_status st = check_common(ko, vo, ki, vi, n, kt, pairs);
  if (st != BCF_OK) return st;
  if (n == 0 || nseg == 0) return BCF_OK;
  if (!off || (reinterpret_cast<uintptr_t>(off) & 7u)) return BCF_EINVAL;
  if (nseg > 0xFFFFFFFFull) return BCF_EUNSUPPORTED;
  const int kb = key_bytes_of(kt);
  const SegLayout wl = seg_layout(n, nseg, kb, pairs);
  st = check_ws(ws, ws_bytes, wl.total, ko, vo, ki, vi, n, kb);
  if (st != BCF_OK) return st;
  uint32_t* err = error_word_ptr();
  if (!err) return BCF_ECUDA;
  char* wsb = static_cast<char*>(ws);
  SegLaunch L{};
  L.kin = ki;
  L.vin = vi;
  L.kout = ko;
  L.vout = vo;
  L.kbuf = wsb + wl.keys;
  L.vbuf = pairs ? reinterpret_cast<uint32_t*>(wsb + wl.vals) : nullptr;
  L.off = off;
  L.nseg = nseg;
  L.n = n;
  L.mode = mode_of(kt, o);
  L.skip_odd = skip_odd ? 1 : 0;
  L.queue = wsb + wl.queue;
  L.capacity = wl.capacity;
  L.items_left = reinterpret_cast<uint32_t*>(wsb + wl.items);
  L.tiny_list = reinterpret_cast<uint32_t*>(wsb + wl.tiny);
  L.tile_base = reinterpret_cast<uint64_t*>(wsb + wl.tbase);
  L.piece_split = reinterpret_cast<uint64_t*>(wsb + wl.splits);
  L.ctl = wsb + wl.ctl;
  L.err = err;
  const SegTuning tu = seg_tuning_for(kb, pairs, n);
  const int cfg = tu.seg_cfg;
  L.merge_cfg = tu.merge_cfg;
  L.order = reinterpret_cast<uint32_t*>(wsb + wl.order);
  L.piece_end = reinterpret_cast<uint64_t*>(wsb + wl.pend);
  L.count_ge = reinterpret_cast<uint32_t*>(wsb + wl.count_ge);
  L.samples_out = wsb + wl.samp0;
  L.samples_buf = wsb + wl.samp1;
  // unpublished queue slots must read "not ready"
  if (cudaMemsetAsync(L.queue, 0, wl.capacity * seg_work_bytes(), s) != cudaSuccess)
    return BCF_ECUDA;
  cudaError_t e = timed(3, s, [&] { return launch_segmented(kb, pairs, cfg, L, s); });
  if (e != cudaSuccess || L.merge_cfg < 0) return from_cuda(e);
  // Merge passes of the listed (multi-tile) segments, by passes to go q: the
  // launch for q does the pass of every segment that has q or more left.
  // The host does not know the longest segment, so q starts at the pass
  // count of a segment of all n keys; launches with no segment that long
  // find no work items and return at once.
  const uint64_t T = static_cast<uint64_t>(kSegCfgs[cfg].tile());
  const uint64_t max_tiles = (n - 1) / T + 2;
  uint32_t qmax = 0;
  while ((1ull << qmax) < max_tiles) ++qmax;
  SegPassList pl{};
  pl.off = off;
  pl.order = L.order;
  pl.piece_end = L.piece_end;
  pl.count_ge = L.count_ge;
  pl.items = reinterpret_cast<SegItem*>(wsb + wl.pitems);
  pl.chunk_seg = reinterpret_cast<uint32_t*>(wsb + wl.chunks);
  pl.next = reinterpret_cast<unsigned long long*>(wsb + wl.pnext);
  pl.n = n;
  pl.T = static_cast<uint32_t>(T);
  e = timed(1, s, [&] { return launch_seg_chunks(pl, s); });
  if (e != cudaSuccess) return BCF_ECUDA;
  for (uint32_t q = qmax; q >= 1; --q) {
    // the last pass (q = 1) writes the output: pass q writes it when q is odd
    const bool to_out = (q & 1u) != 0;
    MergeArgs ma{};
    ma.kin = to_out ? L.kbuf : ko;
    ma.vin = pairs ? (to_out ? L.vbuf : vo) : nullptr;
    ma.kout = to_out ? ko : L.kbuf;
    ma.vout = pairs ? (to_out ? vo : L.vbuf) : nullptr;
    ma.n = n;
    ma.splits = L.piece_split;
    ma.mode_in = 0;  // the block sort left the listed segments' keys mapped
    ma.mode_out = q == 1 ? L.mode : 0;
    // samples of the buffer read (written by the tile sorts or the pass
    // before) and, for a pass with a successor, of the buffer written
    ma.samples_in = to_out ? L.samples_buf : L.samples_out;
    ma.samples_out = q > 1 ? (to_out ? L.samples_out : L.samples_buf) : nullptr;
    ma.err = err;
    pl.q = q;
    e = timed(1, s, [&] { return launch_seg_partition(kb, L.merge_cfg, ma, pl, s); });
    if (e != cudaSuccess) return BCF_ECUDA;
    e = timed(2, s, [&] { return launch_seg_merge(kb, pairs, L.merge_cfg, ma, pl, s); });
    if (e != cudaSuccess) return BCF_ECUDA;
  }
  return BCF_OK;
}

// ---------------------------------------------------------------- pivot buckets

// [header | block-sorted keys | their payloads | samples | sorted samples |
//  workspace of the sample sort | splitters | m | piece sizes | piece offsets |
//  scan workspace | bucket boundaries | segmented-sort workspace]
struct PbLayout {
  size_t xk, xv, samples, ssorted, ssort_ws, ssort_bytes, splitters, nsplit, counts, offsets, cps,
      cps_bytes, seg_off, seg, seg_bytes, total;
  uint64_t ns, ntiles;
  uint32_t T;
};
PbLayout pb_layout(uint64_t n, int kb, bool pairs) {
  PbLayout w;
  const Plan plan = make_plan(n, kb, pairs);
  w.T = plan.T;
  w.ns = (n + kPbSampleStride - 1) / kPbSampleStride;
  w.ntiles = (n + plan.T - 1) / plan.T;
  w.xk = kAlign;
  w.xv = align_up(w.xk + n * kb, kAlign);
  w.samples = align_up(w.xv + (pairs ? n * 4 : 0), kAlign);
  w.ssorted = align_up(w.samples + w.ns * kb, kAlign);
  w.ssort_ws = align_up(w.ssorted + w.ns * kb, kAlign);
  w.ssort_bytes = ws_layout(w.ns, 0, kb, false).total;
  w.splitters = align_up(w.ssort_ws + w.ssort_bytes, kAlign);
  w.nsplit = align_up(w.splitters + kPbSplitters * kb, kAlign);
  w.counts = align_up(w.nsplit + sizeof(uint32_t), kAlign);
  const uint64_t pieces = static_cast<uint64_t>(kPbBuckets) * w.ntiles;
  w.offsets = align_up(w.counts + pieces * 4, kAlign);
  w.cps = align_up(w.offsets + pieces * 4, kAlign);
  w.cps_bytes = kAlign + align_up(((pieces + kCpsTile - 1) / kCpsTile) * 8, kAlign);
  w.seg_off = align_up(w.cps + w.cps_bytes, kAlign);
  w.seg = align_up(w.seg_off + (kPbBuckets + 1) * sizeof(uint64_t), kAlign);
  w.seg_bytes = seg_layout(n, kPbBuckets, kb, pairs).total;
  w.total = align_up(w.seg + w.seg_bytes, kAlign);
  const size_t merge_need = ws_layout(n, 0, kb, pairs).total;  // the fallback's
  if (w.total < merge_need) w.total = merge_need;
  return w;
}

// Pivot buckets pay off once there are several tiles; offsets are 32-bit.
bool pb_applies(uint64_t n, int kb, bool pairs) {
  const Plan plan = make_plan(n, kb, pairs);
  return n > 2ull * plan.T && n < 0xFFFFFFFFull;
}

bcf_status run_sort_pb(void* ko, uint32_t* vo, const void* ki, const uint32_t* vi, uint64_t n,
                       bcf_dtype kt, const bcf_opts* o, void* ws, size_t ws_bytes,
                       cudaStream_t s, bool pairs) {
  bcf_status st = check_common(ko, vo, ki, vi, n, kt, pairs);
  if (st != BCF_OK || n == 0) return st;
  const int kb = key_bytes_of(kt);
  if (!pb_applies(n, kb, pairs)) return run_sort(ko, vo, ki, vi, n, kt, o, ws, ws_bytes, s, pairs);
  const PbLayout wl = pb_layout(n, kb, pairs);
  st = check_ws(ws, ws_bytes, wl.total, ko, vo, ki, vi, n, kb);
  if (st != BCF_OK) return st;
  const int mode = mode_of(kt, o);
  uint32_t* err = error_word_ptr();
  if (!err) return BCF_ECUDA;
  char* wsb = static_cast<char*>(ws);
  const Plan plan = make_plan(n, kb, pairs);

  PbArgs a{};
  a.kin = ki;
  a.n = n;
  a.mode = mode;
  a.samples = wsb + wl.samples;
  a.ns = wl.ns;
  a.sorted_samples = wsb + wl.ssorted;
  a.splitters = wsb + wl.splitters;
  a.nsplit = reinterpret_cast<uint32_t*>(wsb + wl.nsplit);
  a.x = wsb + wl.xk;
  a.xv = pairs ? reinterpret_cast<const uint32_t*>(wsb + wl.xv) : nullptr;
  a.T = wl.T;
  a.ntiles = wl.ntiles;
  a.counts = reinterpret_cast<uint32_t*>(wsb + wl.counts);
  a.offsets = reinterpret_cast<const uint32_t*>(wsb + wl.offsets);
  a.kout = ko;
  a.vout = vo;
  a.seg_off = reinterpret_cast<uint64_t*>(wsb + wl.seg_off);
  a.sample_stride = kPbSampleStride;
  auto step = [&](int which) {
    return from_cuda(timed(5, s, [&] { return launch_pb(which, kb, pairs, a, s); }));
  };

  // 1-2. splitters from a sorted sample of every 256th key (mapped order)
  if ((st = step(kPbStepSample)) != BCF_OK) return st;
  const bcf_dtype ukt = kb == 4 ? BCF_U32 : BCF_U64;  // the samples are mapped already
  st = run_sort(wsb + wl.ssorted, nullptr, wsb + wl.samples, nullptr, wl.ns, ukt, nullptr,
                wsb + wl.ssort_ws, wl.ssort_bytes, s, false);
  if (st != BCF_OK) return st;
  if ((st = step(kPbStepSplitters)) != BCF_OK) return st;
  // 3. block sort into the workspace, keys kept mapped
  BlockSortArgs ba{ki, vi, wsb + wl.xk, pairs ? reinterpret_cast<uint32_t*>(wsb + wl.xv) : nullptr,
                   n, mode, 0, nullptr};
  if (timed(0, s, [&] { return launch_block_sort(kb, pairs, plan.tune.block_cfg, ba, s); }) !=
      cudaSuccess)
    return BCF_ECUDA;
  // 4. piece sizes of every (bucket, tile); 5. their exclusive prefix sum
  if ((st = step(kPbStepCount)) != BCF_OK) return st;
  if (cudaMemsetAsync(wsb + wl.cps, 0, wl.cps_bytes, s) != cudaSuccess) return BCF_ECUDA;
  CpsArgs c{};
  c.out = reinterpret_cast<uint32_t*>(wsb + wl.offsets);
  c.values = a.counts;
  c.colors = nullptr;
  c.n = static_cast<uint64_t>(kPbBuckets) * wl.ntiles;
  c.d = 1;
  c.exclusive = 1;
  c.ntiles = (c.n + kCpsTile - 1) / kCpsTile;
  c.counter = reinterpret_cast<uint32_t*>(wsb + wl.cps);
  c.status = reinterpret_cast<unsigned long long*>(wsb + wl.cps + kAlign);
  c.err = err;
  if (timed(4, s, [&] { return launch_cps(c, 0, s); }) != cudaSuccess) return BCF_ECUDA;
  // 6. every piece to its bucket: equal buckets are final
  if ((st = step(kPbStepScatter)) != BCF_OK) return st;
  if ((st = step(kPbStepSegOffsets)) != BCF_OK) return st;
  // 7. the open buckets, sorted in place (odd = equal buckets skipped)
  return run_segmented(ko, vo, ko, vo, a.seg_off, kPbBuckets, n, kt, o, wsb + wl.seg,
                       wl.seg_bytes, s, true);
}

// BCF_ALGO_AUTO: sample every S-th key, S = n / kAutoMinSamples clamped to
// [kPbSampleStride, kAutoMaxStride], sort the sample, pick splitters from it as
// pivot buckets would, and count the sample keys equal to a splitter beyond
// the splitters' own occurrences (each splitter is a sample key, which alone
// would count 255 of a few hundred samples of distinct keys as equal) -- an
// estimate of the share of keys pivot buckets would leave in final position
// after one distribution.  Pivot buckets when that share reaches
// kAutoEqualNum / kAutoEqualDen, else the merge path.  Measured on GB300 at
// 2^28 keys, with the open buckets on the segmented sort's merge launches:
// pivot buckets take 8.3 ms on distinct keys, 2.9 ms with 16 distinct values
// and 5.9 ms on Zipf(1.1) keys (share 0.5) against 6.7 ms on the merge path,
// a break-even near a share of 0.3 (0.2 with payloads).  The counts are read
// back to the host: the call synchronises `s` once.
constexpr uint32_t kAutoMaxStride = 4096;
constexpr uint64_t kAutoMinSamples = 16384;
constexpr uint32_t kAutoEqualNum = 1, kAutoEqualDen = 3;

bcf_status choose_auto(const void* ki, uint64_t n, bcf_dtype kt, const bcf_opts* o, void* ws,
                       size_t ws_bytes, cudaStream_t s, bool pairs, bool* use_pb) {
  *use_pb = false;
  const int kb = key_bytes_of(kt);
  if (!pb_applies(n, kb, pairs)) return BCF_OK;
  const PbLayout wl = pb_layout(n, kb, pairs);
  if (ws_bytes < wl.total || !ws) return BCF_ENOMEM;
  char* wsb = static_cast<char*>(ws);
  PbArgs a{};
  a.kin = ki;
  a.n = n;
  a.mode = mode_of(kt, o);
  const uint64_t want = n / kAutoMinSamples;
  const uint64_t stride = want > kAutoMaxStride ? kAutoMaxStride : want;
  a.sample_stride = static_cast<uint32_t>(stride < kPbSampleStride ? kPbSampleStride : stride);
  a.ns = (n + a.sample_stride - 1) / a.sample_stride;
  a.samples = wsb + wl.samples;
  a.sorted_samples = wsb + wl.ssorted;
  a.splitters = wsb + wl.splitters;
  a.nsplit = reinterpret_cast<uint32_t*>(wsb + wl.nsplit);
  a.equal_count = reinterpret_cast<uint32_t*>(wsb + wl.counts);
  a.T = wl.T;
  a.ntiles = wl.ntiles;
  auto step = [&](int which) {
    return from_cuda(timed(5, s, [&] { return launch_pb(which, kb, pairs, a, s); }));
  };
  bcf_status st;
  if ((st = step(kPbStepSample)) != BCF_OK) return st;
  const bcf_dtype ukt = kb == 4 ? BCF_U32 : BCF_U64;  // the samples are mapped already
  st = run_sort(wsb + wl.ssorted, nullptr, wsb + wl.samples, nullptr, a.ns, ukt, nullptr,
                wsb + wl.ssort_ws, wl.ssort_bytes, s, false);
  if (st != BCF_OK) return st;
  if ((st = step(kPbStepSplitters)) != BCF_OK) return st;
  if (cudaMemsetAsync(a.equal_count, 0, sizeof(uint32_t), s) != cudaSuccess) return BCF_ECUDA;
  if ((st = step(kPbStepEqualCount)) != BCF_OK) return st;
  uint32_t equal = 0, nsplit = 0;
  if (cudaMemcpyAsync(&equal, a.equal_count, sizeof(equal), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(&nsplit, a.nsplit, sizeof(nsplit), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BCF_ECUDA;
  // the splitters' own occurrences in the sample do not count
  const uint64_t extra = equal > nsplit ? equal - nsplit : 0;
  const uint64_t rest = a.ns > nsplit ? a.ns - nsplit : 0;
  *use_pb = rest > 0 && extra * kAutoEqualDen >= rest * kAutoEqualNum;
  return BCF_OK;
}

// ---------------------------------------------------------------- dispatch

bcf_status sort_any(void* ko, uint32_t* vo, const void* ki, const uint32_t* vi, uint64_t n,
                    bcf_dtype kt, const bcf_opts* o, void* ws, size_t ws_bytes, cudaStream_t s,
                    bool pairs);

// ---------------------------------------------------------------- 16-bit keys

// [header | widened keys in | widened keys out | workspace of the 32-bit call]
struct Wide16Layout {
  size_t kin, kout, inner, total;
};
Wide16Layout wide16_layout(uint64_t n, size_t inner_bytes) {
  Wide16Layout w;
  w.kin = kAlign;
  w.kout = align_up(w.kin + n * 4, kAlign);
  w.inner = align_up(w.kout + n * 4, kAlign);
  w.total = align_up(w.inner + inner_bytes, kAlign);
  return w;
}

// Widens the 16-bit keys [0, n) of `ki`, runs `op(kout32, kin32, inner_ws,
// inner_bytes)` -- the same call on 32-bit keys -- and narrows its output
// [lo, n) into `ko`.  The widening is order-preserving (zero extension for
// u16, sign extension for i16), so the 32-bit result is the 16-bit one.
template <typename Op>
bcf_status via_wide16(void* ko, const void* ki, uint64_t lo, uint64_t n, bcf_dtype kt, void* ws,
                      size_t ws_bytes, size_t inner_bytes, cudaStream_t s, Op op) {
  const Wide16Layout wl = wide16_layout(n, inner_bytes);
  if (ws_bytes < wl.total || !ws) return BCF_ENOMEM;
  if (!aligned16(ws)) return BCF_EINVAL;
  const Span sw{ws, wl.total};
  if (overlap(sw, {ko, n * 2}) || overlap(sw, {ki, n * 2})) return BCF_EINVAL;
  char* wsb = static_cast<char*>(ws);
  uint32_t* kin32 = reinterpret_cast<uint32_t*>(wsb + wl.kin);
  uint32_t* kout32 = reinterpret_cast<uint32_t*>(wsb + wl.kout);
  if (launch_widen16(kin32, static_cast<const uint16_t*>(ki), n, kt == BCF_I16, s) !=
      cudaSuccess)
    return BCF_ECUDA;
  const bcf_status st = op(kout32, kin32, wsb + wl.inner, inner_bytes);
  if (st != BCF_OK) return st;
  if (launch_narrow16(static_cast<uint16_t*>(ko) + lo, kout32 + lo, n - lo, s) != cudaSuccess)
    return BCF_ECUDA;
  return BCF_OK;
}

// The workspace of a device sort of n keys of type kt.
size_t sort_ws_bytes(uint64_t n, bcf_dtype kt, bool pairs, bool pb) {
  if (is16(kt)) return wide16_layout(n, sort_ws_bytes(n, wide_of(kt), pairs, pb)).total;
  const int kb = key_bytes_of(kt);
  return pb ? pb_layout(n, kb, pairs).total : ws_layout(n, 0, kb, pairs).total;
}

// A device sort: merge passes or pivot buckets, any key type.
bcf_status sort_any(void* ko, uint32_t* vo, const void* ki, const uint32_t* vi, uint64_t n,
                    bcf_dtype kt, const bcf_opts* o, void* ws, size_t ws_bytes, cudaStream_t s,
                    bool pairs) {
  bool pb = o && o->algorithm == BCF_ALGO_PIVOT_BUCKETS;
  const bool autom = o && o->algorithm == BCF_ALGO_AUTO;
  if (o && o->algorithm != BCF_ALGO_MERGE && !pb && !autom) return BCF_EINVAL;
  if (autom && !is16(kt)) {
    bcf_status st = check_common(ko, vo, ki, vi, n, kt, pairs);
    if (st != BCF_OK || n == 0) return st;
    st = check_ws(ws, ws_bytes, sort_ws_bytes(n, kt, pairs, true), ko, vo, ki, vi, n,
                  key_bytes_of(kt));
    if (st != BCF_OK) return st;
    if ((st = choose_auto(ki, n, kt, o, ws, ws_bytes, s, pairs, &pb)) != BCF_OK) return st;
  } else if (autom) {
    pb = true;  // 16-bit keys: decided on the widened 32-bit keys below
  }
  if (is16(kt)) {
    bcf_status st = check_common(ko, vo, ki, vi, n, kt, pairs);
    if (st != BCF_OK || n == 0) return st;
    const bcf_dtype wk = wide_of(kt);
    return via_wide16(ko, ki, 0, n, kt, ws, ws_bytes, sort_ws_bytes(n, wk, pairs, pb), s,
                      [&](void* k32o, const void* k32i, void* iw, size_t ib) {
                        return sort_any(k32o, vo, k32i, vi, n, wk, o, iw, ib, s, pairs);
                      });
  }
  if (pb) return run_sort_pb(ko, vo, ki, vi, n, kt, o, ws, ws_bytes, s, pairs);
  return run_sort(ko, vo, ki, vi, n, kt, o, ws, ws_bytes, s, pairs);
}

// ---------------------------------------------------------------- wide payloads

// [header | row indices in | row indices out | workspace of the pairs sort]
struct WideLayout {
  size_t idx_in, idx_out, inner, inner_bytes, total;
};
WideLayout wide_layout(uint64_t n, bcf_dtype kt) {
  WideLayout w;
  w.idx_in = kAlign;
  w.idx_out = align_up(w.idx_in + n * 4, kAlign);
  w.inner = align_up(w.idx_out + n * 4, kAlign);
  const size_t merge = sort_ws_bytes(n, kt, true, false), pb = sort_ws_bytes(n, kt, true, true);
  w.inner_bytes = merge > pb ? merge : pb;  // either algorithm
  w.total = align_up(w.inner + w.inner_bytes, kAlign);
  return w;
}

// Stable sort by key with payload rows of `val_bytes` bytes: the pairs sort of
// (key, row index), then the rows gathered in the sorted order.
bcf_status run_sort_wide(void* ko, void* vo, const void* ki, const void* vi, uint64_t n,
                         uint32_t val_bytes, bcf_dtype kt, const bcf_opts* o, void* ws,
                         size_t ws_bytes, cudaStream_t s) {
  if (!dtype_ok(kt) || val_bytes < 4 || val_bytes % 4 != 0 || val_bytes > 4096) return BCF_EINVAL;
  if (n == 0) return BCF_OK;
  if (!ko || !ki || !vo || !vi) return BCF_EINVAL;
  if (!aligned16(ko) || !aligned16(ki) || (reinterpret_cast<uintptr_t>(vo) & 3u) ||
      (reinterpret_cast<uintptr_t>(vi) & 3u))
    return BCF_EINVAL;
  if (n > 0xFFFFFFFFull) return BCF_EUNSUPPORTED;  // 32-bit row indices
  const size_t kb = key_bytes_of(kt);
  const Span sko{ko, n * kb}, ski{ki, n * kb}, svo{vo, n * val_bytes}, svi{vi, n * val_bytes};
  // the payloads cannot be permuted in place: the gather reads rows in any order
  if (bad_overlap(sko, ski) || overlap(svo, svi) || overlap(sko, svo) || overlap(sko, svi) ||
      overlap(ski, svo))
    return BCF_EINVAL;
  const WideLayout wl = wide_layout(n, kt);
  if (ws_bytes < wl.total || !ws) return BCF_ENOMEM;
  if (!aligned16(ws)) return BCF_EINVAL;
  const Span sw{ws, wl.total};
  if (overlap(sw, sko) || overlap(sw, ski) || overlap(sw, svo) || overlap(sw, svi))
    return BCF_EINVAL;
  char* wsb = static_cast<char*>(ws);
  uint32_t* idx_in = reinterpret_cast<uint32_t*>(wsb + wl.idx_in);
  uint32_t* idx_out = reinterpret_cast<uint32_t*>(wsb + wl.idx_out);
  if (launch_iota(idx_in, n, s) != cudaSuccess) return BCF_ECUDA;
  const bcf_status st =
      sort_any(ko, idx_out, ki, idx_in, n, kt, o, wsb + wl.inner, wl.inner_bytes, s, true);
  if (st != BCF_OK) return st;
  return from_cuda(launch_gather(vo, vi, idx_out, n, val_bytes, s));
}

// ---------------------------------------------------------------- host buffers

// [header | device keys in | values in | keys out | values out | sort workspace]
struct HostLayout {
  size_t kin, vin, kout, vout, sort, sort_bytes, total;
};
size_t sort_ws_bytes(uint64_t n, bcf_dtype kt, bool pairs, bool pb);

HostLayout host_layout(uint64_t n, bcf_dtype kt, bool pairs, bool pb) {
  HostLayout w;
  const int kb = key_bytes_of(kt);
  w.kin = kAlign;
  w.vin = align_up(w.kin + n * kb, kAlign);
  w.kout = align_up(w.vin + (pairs ? n * 4 : 0), kAlign);
  w.vout = align_up(w.kout + n * kb, kAlign);
  w.sort = align_up(w.vout + (pairs ? n * 4 : 0), kAlign);
  w.sort_bytes = sort_ws_bytes(n, kt, pairs, pb);
  w.total = align_up(w.sort + w.sort_bytes, kAlign);
  return w;
}

// One copy stream per device, shared by all host-buffer calls (the copy
// engines are shared anyway), and a pool of timing-free events.  A stream
// wait takes the event's state at the time of the call, so an event can be
// recorded again by a later call.
struct CopyEngine {
  std::mutex mu;
  cudaStream_t stream[64] = {};
  std::vector<cudaEvent_t> events[64];
  size_t next[64] = {};
};
CopyEngine& copy_engine() {
  static CopyEngine c;
  return c;
}
cudaStream_t copy_stream(int dev) {
  CopyEngine& c = copy_engine();
  std::lock_guard<std::mutex> lk(c.mu);
  if (!c.stream[dev] && cudaStreamCreateWithFlags(&c.stream[dev], cudaStreamNonBlocking) !=
                            cudaSuccess)
    c.stream[dev] = nullptr;
  return c.stream[dev];
}
cudaEvent_t copy_event(int dev) {
  constexpr size_t kPool = 64;
  CopyEngine& c = copy_engine();
  std::lock_guard<std::mutex> lk(c.mu);
  auto& ev = c.events[dev];
  if (ev.size() < kPool) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    ev.push_back(e);
    return e;
  }
  return ev[c.next[dev]++ % kPool];
}

struct HostChunks {
  const char* hk;
  const uint32_t* hv;
  char* dk;
  uint32_t* dv;
  uint64_t n, T;
  int kb, dev;
  cudaStream_t cs;
};
// Copies the input of tiles [t0, t1) on the copy stream and makes `s` wait
// for it.
bcf_status copy_in_tiles(void* ctx, uint64_t t0, uint64_t t1, cudaStream_t s) {
  HostChunks& h = *static_cast<HostChunks*>(ctx);
  const uint64_t off = t0 * h.T, end = t1 * h.T < h.n ? t1 * h.T : h.n;
  if (cudaMemcpyAsync(h.dk + off * h.kb, h.hk + off * h.kb, (end - off) * h.kb,
                      cudaMemcpyHostToDevice, h.cs) != cudaSuccess)
    return BCF_ECUDA;
  if (h.hv && cudaMemcpyAsync(h.dv + off, h.hv + off, (end - off) * 4, cudaMemcpyHostToDevice,
                              h.cs) != cudaSuccess)
    return BCF_ECUDA;
  cudaEvent_t ev = copy_event(h.dev);
  if (!ev || cudaEventRecord(ev, h.cs) != cudaSuccess || cudaStreamWaitEvent(s, ev, 0) != cudaSuccess)
    return BCF_ECUDA;
  return BCF_OK;
}

bcf_status run_sort_host(void* hko, uint32_t* hvo, const void* hki, const uint32_t* hvi,
                         uint64_t n, bcf_dtype kt, const bcf_opts* o, void* ws, size_t ws_bytes,
                         cudaStream_t s, bool pairs) {
  if (!dtype_ok(kt)) return BCF_EINVAL;
  if (n == 0) return BCF_OK;
  if (!hko || !hki || (pairs && (!hvo || !hvi))) return BCF_EINVAL;
  const int kb = key_bytes_of(kt);
  // the automatic choice is made by the device sort below, on the copied-in
  // keys: it needs the pivot-bucket workspace and the whole input first
  const bool pb = o && (o->algorithm == BCF_ALGO_PIVOT_BUCKETS || o->algorithm == BCF_ALGO_AUTO);
  if (o && o->algorithm != BCF_ALGO_MERGE && !pb) return BCF_EINVAL;
  const HostLayout wl = host_layout(n, kt, pairs, pb);
  if (ws_bytes < wl.total || !ws) return BCF_ENOMEM;
  if (!aligned16(ws)) return BCF_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BCF_ECUDA;
  char* wsb = static_cast<char*>(ws);
  char* dki = wsb + wl.kin;
  uint32_t* dvi = pairs ? reinterpret_cast<uint32_t*>(wsb + wl.vin) : nullptr;
  char* dko = wsb + wl.kout;
  uint32_t* dvo = pairs ? reinterpret_cast<uint32_t*>(wsb + wl.vout) : nullptr;
  bcf_status st;
  if (pb || is16(kt)) {  // the whole input first (one copy in), then the device sort
    if (cudaMemcpyAsync(dki, hki, n * kb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (pairs && cudaMemcpyAsync(dvi, hvi, n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess))
      return BCF_ECUDA;
    st = sort_any(dko, dvo, dki, dvi, n, kt, o, wsb + wl.sort, wl.sort_bytes, s, pairs);
  } else {
    // copy in on the copy stream, in 8 pieces of whole tiles; each piece's
    // block sort starts as soon as it has landed
    cudaStream_t cs = copy_stream(dev);
    cudaEvent_t start = copy_event(dev);
    if (!cs || !start || cudaEventRecord(start, s) != cudaSuccess ||
        cudaStreamWaitEvent(cs, start, 0) != cudaSuccess)  // the workspace is free by then
      return BCF_ECUDA;
    const Plan plan = make_plan(n, kb, pairs);
    const uint64_t tiles = (n + plan.T - 1) / plan.T;
    HostChunks h{static_cast<const char*>(hki), hvi, dki, dvi, n, plan.T, kb, dev, cs};
    ChunkedInput ci{(tiles + 7) / 8, copy_in_tiles, &h};
    st = run_sort(dko, dvo, dki, dvi, n, kt, o, wsb + wl.sort, wl.sort_bytes, s, pairs, &ci);
  }
  if (st != BCF_OK) return st;
  if (cudaMemcpyAsync(hko, dko, n * kb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      (pairs && cudaMemcpyAsync(hvo, dvo, n * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess))
    return BCF_ECUDA;
  return BCF_OK;
}

// ---------------------------------------------------------------- colored prefix sums

struct CpsLayout {
  size_t counter, status, total;
  uint64_t ntiles;
};
CpsLayout cps_layout(uint64_t n, uint32_t d) {
  CpsLayout w;
  w.ntiles = (n + kCpsTile - 1) / kCpsTile;
  w.counter = 0;
  w.status = kAlign;
  w.total = align_up(w.status + w.ntiles * d * sizeof(unsigned long long), kAlign);
  return w;
}

bcf_status run_cps(uint32_t* out, const uint32_t* values, const uint8_t* colors, uint64_t n,
                   uint32_t d, int exclusive, int layout, void* ws, size_t ws_bytes,
                   cudaStream_t s) {
  if (d < 1 || d > kCpsMaxColors || (layout != BCF_CPS_BANKED && layout != BCF_CPS_ROWS))
    return BCF_EINVAL;
  if (n == 0) return BCF_OK;
  if (!out || !values || !colors) return BCF_EINVAL;
  if (!aligned16(out) || !aligned16(values) || !aligned16(colors)) return BCF_EINVAL;
  if (n > (1ull << 42)) return BCF_EUNSUPPORTED;
  const Span so{out, n * 4}, sv{values, n * 4}, sc{colors, n};
  if (bad_overlap(so, sv) || overlap(so, sc)) return BCF_EINVAL;
  const CpsLayout wl = cps_layout(n, d);
  if (ws_bytes < wl.total || !ws) return BCF_ENOMEM;
  if (!aligned16(ws)) return BCF_EINVAL;
  const Span sw{ws, wl.total};
  if (overlap(sw, so) || overlap(sw, sv) || overlap(sw, sc)) return BCF_EINVAL;
  uint32_t* err = error_word_ptr();
  if (!err) return BCF_ECUDA;
  // tile ticket and every status word start at zero ("nothing published")
  if (cudaMemsetAsync(ws, 0, wl.total, s) != cudaSuccess) return BCF_ECUDA;
  char* wsb = static_cast<char*>(ws);
  CpsArgs a{};
  a.out = out;
  a.values = values;
  a.colors = colors;
  a.n = n;
  a.d = d;
  a.exclusive = exclusive ? 1 : 0;
  a.ntiles = wl.ntiles;
  a.status = reinterpret_cast<unsigned long long*>(wsb + wl.status);
  a.counter = reinterpret_cast<uint32_t*>(wsb + wl.counter);
  a.err = err;
  const cudaError_t e = timed(4, s, [&] { return launch_cps(a, layout, s); });
  return from_cuda(e);
}

}  // namespace
}  // namespace bcf

// ==================================================================== C ABI

using namespace bcf;

extern "C" {

size_t bcf_workspace_bytes(int op, uint64_t n, uint64_t nseg_or_k, bcf_dtype kt, int has_vals) {
  if (!dtype_ok(kt)) return 0;
  const bool pairs = has_vals != 0;
  if (is16(kt)) {  // 16-bit keys: widened copies in and out, then the 32-bit call's workspace
    const bcf_dtype wk = wide_of(kt);
    switch (op) {
      case BCF_OP_SORT:
      case BCF_OP_MERGE:
      case BCF_OP_SEGMENTED:
      case BCF_OP_SORT_PB:
        return wide16_layout(n, bcf_workspace_bytes(op, n, nseg_or_k, wk, has_vals)).total;
      case BCF_OP_SORT_HOST: return host_layout(n, kt, pairs, false).total;
      case BCF_OP_SORT_HOST_PB: return host_layout(n, kt, pairs, true).total;
      case BCF_OP_SORT_WIDE: return wide_layout(n, kt).total;
      default: return 0;
    }
  }
  const int kb = key_bytes_of(kt);
  switch (op) {
    case BCF_OP_SORT: return ws_layout(n, 0, kb, pairs).total;
    case BCF_OP_MERGE: return ws_layout(n, nseg_or_k, kb, pairs).total;
    case BCF_OP_SEGMENTED: return seg_layout(n, nseg_or_k, kb, pairs).total;
    case BCF_OP_SORT_PB: return pb_layout(n, kb, pairs).total;
    case BCF_OP_SORT_HOST: return host_layout(n, kt, pairs, false).total;
    case BCF_OP_SORT_HOST_PB: return host_layout(n, kt, pairs, true).total;
    case BCF_OP_SORT_WIDE: return wide_layout(n, kt).total;
    case BCF_OP_CPS:
      if (kt != BCF_U32 || has_vals || nseg_or_k < 1 || nseg_or_k > kCpsMaxColors) return 0;
      return cps_layout(n, static_cast<uint32_t>(nseg_or_k)).total;
    default: return 0;
  }
}

bcf_status bcf_sort_keys(void* keys_out, const void* keys_in, uint64_t n, bcf_dtype kt,
                         const bcf_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream) {
  return sort_any(keys_out, nullptr, keys_in, nullptr, n, kt, opts, ws, ws_bytes, stream, false);
}

bcf_status bcf_sort_pairs(void* keys_out, uint32_t* vals_out, const void* keys_in,
                          const uint32_t* vals_in, uint64_t n, bcf_dtype kt,
                          const bcf_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream) {
  return sort_any(keys_out, vals_out, keys_in, vals_in, n, kt, opts, ws, ws_bytes, stream, true);
}

bcf_status bcf_merge_runs(void* keys_out, uint32_t* vals_out, const void* keys_in,
                          const uint32_t* vals_in, const uint64_t* run_offsets_host, uint32_t k,
                          bcf_dtype kt, const bcf_opts* opts, void* ws, size_t ws_bytes,
                          cudaStream_t stream) {
  if ((vals_out == nullptr) != (vals_in == nullptr)) return BCF_EINVAL;
  if (is16(kt)) {
    if (!run_offsets_host || k == 0) return BCF_EINVAL;
    for (uint32_t r = 0; r < k; ++r)
      if (run_offsets_host[r + 1] < run_offsets_host[r]) return BCF_EINVAL;
    const uint64_t n = run_offsets_host[k], lo = run_offsets_host[0];
    const bool pairs = vals_out != nullptr;
    bcf_status st = check_common(keys_out, vals_out, keys_in, vals_in, n, kt, pairs);
    if (st != BCF_OK || n == lo) return st;
    const bcf_dtype wk = wide_of(kt);
    return via_wide16(keys_out, keys_in, lo, n, kt, ws, ws_bytes,
                      ws_layout(n, k, 4, pairs).total, stream,
                      [&](void* k32o, const void* k32i, void* iw, size_t ib) {
                        return run_merge(k32o, vals_out, k32i, vals_in, run_offsets_host, k, wk,
                                         opts, iw, ib, stream);
                      });
  }
  return run_merge(keys_out, vals_out, keys_in, vals_in, run_offsets_host, k, kt, opts, ws,
                   ws_bytes, stream);
}

bcf_status bcf_segmented_sort(void* keys_out, uint32_t* vals_out, const void* keys_in,
                              const uint32_t* vals_in, const uint64_t* seg_offsets_dev,
                              uint64_t nseg, uint64_t n_total, bcf_dtype kt,
                              const bcf_opts* opts, void* ws, size_t ws_bytes,
                              cudaStream_t stream) {
  if ((vals_out == nullptr) != (vals_in == nullptr)) return BCF_EINVAL;
  if (is16(kt)) {
    const bool pairs = vals_out != nullptr;
    bcf_status st = check_common(keys_out, vals_out, keys_in, vals_in, n_total, kt, pairs);
    if (st != BCF_OK || n_total == 0 || nseg == 0) return st;
    const bcf_dtype wk = wide_of(kt);
    return via_wide16(keys_out, keys_in, 0, n_total, kt, ws, ws_bytes,
                      seg_layout(n_total, nseg, 4, pairs).total, stream,
                      [&](void* k32o, const void* k32i, void* iw, size_t ib) {
                        return run_segmented(k32o, vals_out, k32i, vals_in, seg_offsets_dev, nseg,
                                             n_total, wk, opts, iw, ib, stream);
                      });
  }
  return run_segmented(keys_out, vals_out, keys_in, vals_in, seg_offsets_dev, nseg, n_total, kt,
                       opts, ws, ws_bytes, stream);
}

bcf_status bcf_sort_pairs_wide(void* keys_out, void* vals_out, const void* keys_in,
                               const void* vals_in, uint64_t n, uint32_t val_bytes, bcf_dtype kt,
                               const bcf_opts* opts, void* ws, size_t ws_bytes,
                               cudaStream_t stream) {
  return run_sort_wide(keys_out, vals_out, keys_in, vals_in, n, val_bytes, kt, opts, ws, ws_bytes,
                       stream);
}

bcf_status bcf_sort_keys_host(void* keys_out_host, const void* keys_in_host, uint64_t n,
                              bcf_dtype kt, const bcf_opts* opts, void* ws, size_t ws_bytes,
                              cudaStream_t stream) {
  return run_sort_host(keys_out_host, nullptr, keys_in_host, nullptr, n, kt, opts, ws, ws_bytes,
                       stream, false);
}

bcf_status bcf_sort_pairs_host(void* keys_out_host, uint32_t* vals_out_host,
                               const void* keys_in_host, const uint32_t* vals_in_host, uint64_t n,
                               bcf_dtype kt, const bcf_opts* opts, void* ws, size_t ws_bytes,
                               cudaStream_t stream) {
  return run_sort_host(keys_out_host, vals_out_host, keys_in_host, vals_in_host, n, kt, opts, ws,
                       ws_bytes, stream, true);
}

bcf_status bcf_colored_prefix_sums(uint32_t* out, const uint32_t* values, const uint8_t* colors,
                                   uint64_t n, uint32_t d, int exclusive, int layout, void* ws,
                                   size_t ws_bytes, cudaStream_t stream) {
  return run_cps(out, values, colors, n, d, exclusive, layout, ws, ws_bytes, stream);
}

const char* bcf_status_string(bcf_status s) {
  switch (s) {
    case BCF_OK: return "BCF_OK";
    case BCF_EINVAL: return "BCF_EINVAL: invalid argument";
    case BCF_ENOMEM: return "BCF_ENOMEM: workspace too small";
    case BCF_ECUDA: return "BCF_ECUDA: CUDA error";
    case BCF_ETIMEOUT: return "BCF_ETIMEOUT: device-side wait ran out";
    case BCF_EUNSUPPORTED: return "BCF_EUNSUPPORTED: not supported by this library";
    default: return "BCF: unknown status";
  }
}

bcf_status bcf_last_device_error(cudaStream_t stream) {
  if (cudaStreamSynchronize(stream) != cudaSuccess) return BCF_ECUDA;
  uint32_t v = 0;
  if (cudaMemcpyFromSymbol(&v, g_error_word, sizeof(v)) != cudaSuccess) return BCF_ECUDA;
  if (v != 0) {
    const uint32_t zero = 0;
    if (cudaMemcpyToSymbol(g_error_word, &zero, sizeof(zero)) != cudaSuccess) return BCF_ECUDA;
    // a color >= d alone is an invalid argument; any other bit is a wait that ran out
    return v == kErrBadColor ? BCF_EINVAL : BCF_ETIMEOUT;
  }
  return BCF_OK;
}

__device__ uint32_t g_never_set;  // a flag no code writes: the self-test's wait runs out

static __device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

static __global__ void bounded_wait_selftest_kernel(uint64_t limit_ns, uint32_t* err) {
  if (threadIdx.x != 0) return;
  const volatile uint32_t* flag = &g_never_set;
  const uint64_t t0 = now_ns();
  while (*flag == 0) {
    if (now_ns() - t0 > limit_ns) {
      atomicOr(err, kErrSelftestTimeout);
      return;
    }
    __nanosleep(1000);
  }
}

bcf_status bcf_selftest_bounded_wait(uint32_t limit_us, cudaStream_t stream) {
  if (limit_us == 0 || limit_us > 2000000u) return BCF_EINVAL;
  uint32_t* err = error_word_ptr();
  if (!err) return BCF_ECUDA;
  bounded_wait_selftest_kernel<<<1, 32, 0, stream>>>(static_cast<uint64_t>(limit_us) * 1000u, err);
  return cudaGetLastError() == cudaSuccess ? BCF_OK : BCF_ECUDA;
}

bcf_status bcf_set_wait_limit_us(uint32_t limit_us) {
  if (limit_us > kMaxWaitLimitUs) return BCF_EINVAL;
  g_wait_limit_ns.store(limit_us == 0 ? kDefaultWaitLimitNs : uint64_t(limit_us) * 1000u,
                        std::memory_order_relaxed);
  return BCF_OK;
}

uint32_t bcf_wait_limit_us(void) {
  return static_cast<uint32_t>(g_wait_limit_ns.load(std::memory_order_relaxed) / 1000u);
}

bcf_status bcf_selftest_segmented_wait(void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (ws_bytes < kSegSelftestBytes || !ws) return BCF_ENOMEM;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return BCF_EINVAL;
  uint32_t* err = error_word_ptr();
  if (!err) return BCF_ECUDA;
  return from_cuda(launch_segmented_wait_selftest(ws, wait_limit_ns(), err, stream));
}

bcf_status bcf_profile_set_smem_floor(uint32_t bytes) {
  if (bytes > kMaxSmemFloor) return BCF_EINVAL;
  g_smem_floor.store(bytes, std::memory_order_relaxed);
  return BCF_OK;
}

bcf_status bcf_sort_plan(uint64_t n, bcf_dtype kt, int has_vals, bcf_plan* out) {
  if (!out || !dtype_ok(kt)) return BCF_EINVAL;
  if (is16(kt)) kt = wide_of(kt);  // the passes run on the widened keys
  const int kb = key_bytes_of(kt);
  const Plan p = make_plan(n, kb, has_vals != 0);
  out->block_tile = p.T;
  out->merge_tile = p.Tm;
  out->merge_passes = p.passes;
  out->launches = n == 0 ? 0 : 1 + 2 * p.passes;
  out->bytes_per_pass = 2ull * n * (kb + (has_vals ? 4 : 0));
  return BCF_OK;
}

bcf_status bcf_profile_enable(int on) {
  Profiler& P = prof();
  std::lock_guard<std::mutex> lk(P.mu);
  P.on = on != 0;
  g_profiling.store(P.on, std::memory_order_relaxed);
  return BCF_OK;
}

bcf_status bcf_profile_collect_launches(bcf_profile* out, int* kinds, float* ms_out,
                                        uint32_t max, uint32_t* count) {
  if (!out || !count || (max > 0 && (!kinds || !ms_out))) return BCF_EINVAL;
  Profiler& P = prof();
  std::lock_guard<std::mutex> lk(P.mu);
  bcf_status st = BCF_OK;
  uint32_t i = 0;
  for (auto& r : P.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
      st = BCF_ECUDA;
    if (r.kind >= 0 && r.kind < BCF_PROFILE_KINDS) {
      out->launches[r.kind] += 1;
      out->total_ms[r.kind] += ms;
    }
    if (i < max) {
      kinds[i] = r.kind;
      ms_out[i] = ms;
    }
    ++i;
    P.pool.push_back(r.a);
    P.pool.push_back(r.b);
  }
  *count = i;
  P.pending.clear();
  return st;
}

bcf_status bcf_profile_collect(bcf_profile* out) {
  uint32_t count = 0;
  return bcf_profile_collect_launches(out, nullptr, nullptr, 0, &count);
}

const char* bcf_version(void) { return "bcfsort 0.1 (sm_103a)"; }

bcf_status bcf_tuning_set(const bcf_tuning_entry* entries, int count) {
  if (count == -1) {  // back to the package's table file, read again on next use
    TuneTable& t = tune_table();
    std::lock_guard<std::mutex> lk(t.mu);
    t.rows.clear();
    t.loaded = false;
    return BCF_OK;
  }
  if (count < 0 || (count > 0 && !entries)) return BCF_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!entry_ok(entries[i])) return BCF_EINVAL;
  TuneTable& t = tune_table();
  std::lock_guard<std::mutex> lk(t.mu);
  t.rows.assign(entries, entries + count);
  t.loaded = true;
  return BCF_OK;
}

int bcf_tuning_config(int kind, int index, int* elems_per_thread, int* threads) {
  const TileCfg* tab = kind == 0 ? kBlockCfgs : kind == 1 ? kMergeCfgs : kind == 2 ? kSegCfgs : nullptr;
  const int count = kind == 0 ? kNumBlockCfgs : kind == 1 ? kNumMergeCfgs : kind == 2 ? kNumSegCfgs : 0;
  if (!tab || index < 0 || index >= count) return 0;
  if (elems_per_thread) *elems_per_thread = tab[index].E;
  if (threads) *threads = tab[index].NT;
  return 1;
}

int bcf_tuning_supported(int kind, int index, int key_bytes, int has_vals) {
  switch (kind) {
    case 0: return block_cfg_supported(key_bytes, has_vals != 0, index) ? 1 : 0;
    case 1: return merge_cfg_supported(key_bytes, has_vals != 0, index) ? 1 : 0;
    case 2: return seg_cfg_supported(key_bytes, has_vals != 0, index) ? 1 : 0;
    default: return 0;
  }
}

}  // extern "C"
