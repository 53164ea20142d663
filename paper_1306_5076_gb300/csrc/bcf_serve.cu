// bcf_serve.cu -- continuous-batching request server for sort and merge
// requests (the serving extension of the library; the paper measures one
// sort at a time, Sec. 4).
//
// The caller owns a device arena and drives the server from one host thread:
//   submit()  queues a request (host bookkeeping only);
//   step()    reaps finished work (event polling), frees its arena space,
//             then admits queued requests by memory and launches them;
//   poll()    hands back completion records (submit / admit / done times).
// Served mode (continuous batching): requests up to `small_max` keys that are
// waiting together are coalesced -- per (key type, order, payload) -- into one
// segmented-sort launch over a packed batch in the arena (a lone one runs on
// its own) (a merge of sorted runs is the
// stable sort of their concatenation, so small merges batch the same way);
// larger requests run as their own sort / merge chain with the workspace in
// the arena, round-robin over parallel streams.  Small requests may overtake
// a large one that does not fit yet, so a big request never blocks the queue.
// New arrivals are admitted on every step while earlier work is still on the
// GPU, and their work overlaps on the device.
// Plain mode (the baseline): every request is its own launch chain, in
// arrival order, on one stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "bcfsort.h"

namespace {

constexpr uint64_t kAlignB = 256;
constexpr uint64_t align_up(uint64_t x) { return (x + kAlignB - 1) / kAlignB * kAlignB; }

// ---------------------------------------------------------------- arena allocator

// First-fit allocator over [0, bytes) with a coalescing free list.  Live
// allocations are tracked so that a free must name one exactly (a double free
// or a wrong range is refused instead of corrupting the free list).
struct Arena {
  uint64_t bytes = 0, used = 0, peak = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> size
  std::map<uint64_t, uint64_t> live_;  // offset -> size (rounded)

  void init(uint64_t b) {
    bytes = b / kAlignB * kAlignB;
    used = peak = 0;
    free_.clear();
    live_.clear();
    if (bytes) free_[0] = bytes;
  }
  bool alloc(uint64_t sz, uint64_t* off) {
    sz = align_up(sz ? sz : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= sz) {
        *off = it->first;
        const uint64_t rest = it->second - sz;
        const uint64_t next = it->first + sz;
        free_.erase(it);
        if (rest) free_[next] = rest;
        live_[*off] = sz;
        used += sz;
        if (used > peak) peak = used;
        return true;
      }
    }
    return false;
  }
  // false (nothing changed) unless [off, off + sz) is a live allocation
  bool release(uint64_t off, uint64_t sz) {
    sz = align_up(sz ? sz : 1);
    auto lv = live_.find(off);
    if (lv == live_.end() || lv->second != sz) return false;
    live_.erase(lv);
    used -= sz;
    auto it = free_.emplace(off, sz).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
    return true;
  }
  uint64_t largest_free() const {
    uint64_t m = 0;
    for (auto& kv : free_) m = kv.second > m ? kv.second : m;
    return m;
  }
};

// ---------------------------------------------------------------- batch copy kernels

struct CopyDesc {
  const void* kin;
  const uint32_t* vin;
  void* kout;
  uint32_t* vout;
  uint64_t n, off;  // keys, and the request's first index in the batch
};

// One CTA per request: copy its keys (+ values) into the packed batch
// (gather) or back out to the request's buffers (scatter).
template <bool GATHER>
__global__ void batch_copy_kernel(const CopyDesc* d, void* batch_k, uint32_t* batch_v, int kb) {
  const CopyDesc c = d[blockIdx.x];
  const uint64_t n = c.n;
  if (kb == 4) {
    uint32_t* bk = static_cast<uint32_t*>(batch_k) + c.off;
    const uint32_t* src = GATHER ? static_cast<const uint32_t*>(c.kin) : bk;
    uint32_t* dst = GATHER ? bk : static_cast<uint32_t*>(c.kout);
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  } else if (kb == 2) {
    uint16_t* bk = static_cast<uint16_t*>(batch_k) + c.off;
    const uint16_t* src = GATHER ? static_cast<const uint16_t*>(c.kin) : bk;
    uint16_t* dst = GATHER ? bk : static_cast<uint16_t*>(c.kout);
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  } else {
    uint64_t* bk = static_cast<uint64_t*>(batch_k) + c.off;
    const uint64_t* src = GATHER ? static_cast<const uint64_t*>(c.kin) : bk;
    uint64_t* dst = GATHER ? bk : static_cast<uint64_t*>(c.kout);
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  }
  if (batch_v && c.vin) {
    uint32_t* bv = batch_v + c.off;
    const uint32_t* src = GATHER ? c.vin : bv;
    uint32_t* dst = GATHER ? bv : c.vout;
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  }
}

// ---------------------------------------------------------------- server

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Req {
  bcf_request r;
  std::vector<uint64_t> runs;  // merge: run offsets (relative to the request)
  double t_submit = 0, t_admit = 0;
};

struct Unit {
  cudaEvent_t ev = nullptr;
  std::vector<Req> reqs;
  uint64_t off = 0, bytes = 0;
  int slot = -1;  // pinned staging slot (batches)
};

constexpr int kStagingSlots = 64;
constexpr uint32_t kMaxBatchSegs = 4096;
constexpr size_t kSlotBytes =
    align_up((kMaxBatchSegs + 1) * sizeof(uint64_t)) + align_up(kMaxBatchSegs * sizeof(CopyDesc));

}  // namespace

struct bcf_server {
  bcf_server_config cfg{};
  Arena arena;
  std::vector<cudaStream_t> streams;
  int next_stream = 0;
  std::deque<Req> pending;
  std::vector<Unit> inflight;
  std::vector<bcf_completion> done;
  std::vector<cudaEvent_t> events;
  std::vector<int> free_slots;
  unsigned char* staging = nullptr;  // pinned host, kStagingSlots x kSlotBytes
  std::chrono::steady_clock::time_point t0;
  uint64_t launched_units = 0, launched_batches = 0;
};

namespace {

bcf_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? BCF_OK : BCF_ECUDA; }

int key_bytes(bcf_dtype kt) {
  if (kt == BCF_U16 || kt == BCF_I16) return 2;
  return (kt == BCF_U64 || kt == BCF_I64 || kt == BCF_F64) ? 8 : 4;
}

cudaEvent_t get_event(bcf_server* s) {
  if (!s->events.empty()) {
    cudaEvent_t e = s->events.back();
    s->events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

bool is_small(const bcf_server* s, const Req& q) { return q.r.n <= s->cfg.small_max; }

// Arena bytes a request needs when it runs on its own.
uint64_t solo_bytes(const Req& q) {
  const int op = q.r.op == BCF_OP_MERGE ? BCF_OP_MERGE : BCF_OP_SORT;
  const uint64_t k = q.r.op == BCF_OP_MERGE ? q.r.k : 0;
  return bcf_workspace_bytes(op, q.r.n, k, q.r.kt, q.r.vals_in != nullptr);
}

bcf_status launch_solo(bcf_server* s, Req q, cudaStream_t st) {
  const uint64_t need = solo_bytes(q);
  uint64_t off = 0;
  if (!s->arena.alloc(need, &off)) return BCF_ENOMEM;
  Unit u;
  u.off = off;
  u.bytes = need;
  void* ws = static_cast<char*>(s->cfg.arena) + off;
  bcf_opts o{q.r.descending, 1};
  bcf_status st2;
  if (q.r.op == BCF_OP_MERGE)
    st2 = bcf_merge_runs(q.r.keys_out, q.r.vals_out, q.r.keys_in, q.r.vals_in, q.runs.data(),
                         q.r.k, q.r.kt, &o, ws, need, st);
  else if (q.r.vals_in)
    st2 = bcf_sort_pairs(q.r.keys_out, q.r.vals_out, q.r.keys_in, q.r.vals_in, q.r.n, q.r.kt, &o,
                         ws, need, st);
  else
    st2 = bcf_sort_keys(q.r.keys_out, q.r.keys_in, q.r.n, q.r.kt, &o, ws, need, st);
  u.ev = get_event(s);
  cudaEventRecord(u.ev, st);
  q.t_admit = now_s(s->t0);
  if (st2 != BCF_OK) {
    // the request failed on the host side: report it, release its space
    bcf_completion c{q.r.tag, st2, q.t_submit, q.t_admit, q.t_admit};
    s->done.push_back(c);
    s->arena.release(off, need);
    s->events.push_back(u.ev);
    return BCF_OK;
  }
  u.reqs.push_back(q);
  s->inflight.push_back(std::move(u));
  ++s->launched_units;
  return BCF_OK;
}

// Packed batch: [keys | values | offsets (nseg+1) | descriptors | segmented ws]
bcf_status launch_batch(bcf_server* s, std::vector<Req>& group, cudaStream_t st) {
  if (group.empty()) return BCF_OK;
  if (s->free_slots.empty()) return BCF_ENOMEM;
  const bcf_dtype kt = group[0].r.kt;
  const bool pairs = group[0].r.vals_in != nullptr;
  const int kb = key_bytes(kt);
  uint64_t N = 0;
  for (auto& q : group) N += q.r.n;
  const uint32_t nseg = static_cast<uint32_t>(group.size());
  const uint64_t o_keys = 0;
  const uint64_t o_vals = align_up(N * kb);
  const uint64_t o_offs = o_vals + (pairs ? align_up(N * 4) : 0);
  const uint64_t o_desc = o_offs + align_up((nseg + 1) * sizeof(uint64_t));
  const uint64_t o_ws = o_desc + align_up(nseg * sizeof(CopyDesc));
  const uint64_t ws_bytes = bcf_workspace_bytes(BCF_OP_SEGMENTED, N, nseg, kt, pairs);
  const uint64_t need = o_ws + ws_bytes;
  uint64_t off = 0;
  if (!s->arena.alloc(need, &off)) return BCF_ENOMEM;
  const int slot = s->free_slots.back();
  s->free_slots.pop_back();
  unsigned char* host = s->staging + static_cast<size_t>(slot) * kSlotBytes;
  uint64_t* h_offs = reinterpret_cast<uint64_t*>(host);
  CopyDesc* h_desc = reinterpret_cast<CopyDesc*>(host + align_up((kMaxBatchSegs + 1) * sizeof(uint64_t)));
  uint64_t pos = 0;
  for (uint32_t i = 0; i < nseg; ++i) {
    const Req& q = group[i];
    h_offs[i] = pos;
    h_desc[i] = CopyDesc{q.r.keys_in, q.r.vals_in, q.r.keys_out, q.r.vals_out, q.r.n, pos};
    pos += q.r.n;
  }
  h_offs[nseg] = pos;
  char* base = static_cast<char*>(s->cfg.arena) + off;
  void* bk = base + o_keys;
  uint32_t* bv = pairs ? reinterpret_cast<uint32_t*>(base + o_vals) : nullptr;
  uint64_t* d_offs = reinterpret_cast<uint64_t*>(base + o_offs);
  CopyDesc* d_desc = reinterpret_cast<CopyDesc*>(base + o_desc);
  bcf_status rc = BCF_OK;
  if (cudaMemcpyAsync(d_offs, h_offs, (nseg + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(d_desc, h_desc, nseg * sizeof(CopyDesc), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    rc = BCF_ECUDA;
  if (rc == BCF_OK) {
    batch_copy_kernel<true><<<nseg, 256, 0, st>>>(d_desc, bk, bv, kb);
    rc = cuda_ok(cudaGetLastError());
  }
  bcf_opts o{group[0].r.descending, 1};
  if (rc == BCF_OK)
    rc = bcf_segmented_sort(bk, bv, bk, bv, d_offs, nseg, N, kt, &o, base + o_ws, ws_bytes, st);
  if (rc == BCF_OK) {
    batch_copy_kernel<false><<<nseg, 256, 0, st>>>(d_desc, bk, bv, kb);
    rc = cuda_ok(cudaGetLastError());
  }
  Unit u;
  u.off = off;
  u.bytes = need;
  u.slot = slot;
  u.ev = get_event(s);
  cudaEventRecord(u.ev, st);
  const double t = now_s(s->t0);
  for (auto& q : group) {
    q.t_admit = t;
    if (rc != BCF_OK) {
      s->done.push_back(bcf_completion{q.r.tag, rc, q.t_submit, t, t});
    }
  }
  if (rc != BCF_OK) {
    // nothing to wait for: release once the stream passed the event
    cudaEventSynchronize(u.ev);
    s->arena.release(off, need);
    s->free_slots.push_back(slot);
    s->events.push_back(u.ev);
    return rc;
  }
  u.reqs = std::move(group);
  s->inflight.push_back(std::move(u));
  ++s->launched_units;
  ++s->launched_batches;
  return BCF_OK;
}

void reap(bcf_server* s) {
  const double t = now_s(s->t0);
  for (size_t i = 0; i < s->inflight.size();) {
    Unit& u = s->inflight[i];
    const cudaError_t q = cudaEventQuery(u.ev);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    const bcf_status st = q == cudaSuccess ? BCF_OK : BCF_ECUDA;
    for (auto& r : u.reqs) s->done.push_back(bcf_completion{r.r.tag, st, r.t_submit, r.t_admit, t});
    s->arena.release(u.off, u.bytes);
    if (u.slot >= 0) s->free_slots.push_back(u.slot);
    s->events.push_back(u.ev);
    u = std::move(s->inflight.back());
    s->inflight.pop_back();
  }
}

cudaStream_t pick_stream(bcf_server* s) {
  cudaStream_t st = s->streams[s->next_stream];
  s->next_stream = (s->next_stream + 1) % static_cast<int>(s->streams.size());
  return st;
}

void admit_plain(bcf_server* s) {
  while (!s->pending.empty()) {
    Req q = s->pending.front();
    if (launch_solo(s, q, s->streams[0]) == BCF_ENOMEM) break;
    s->pending.pop_front();
  }
}

void admit_served(bcf_server* s) {
  // groups of coalescable small requests, keyed by (key type, order, payload)
  struct Group {
    bcf_dtype kt;
    int desc;
    bool pairs;
    std::vector<Req> reqs;
    uint64_t keys = 0;
  };
  std::vector<Group> groups;
  std::deque<Req> keep;
  bool large_blocked = false;
  while (!s->pending.empty()) {
    Req q = std::move(s->pending.front());
    s->pending.pop_front();
    if (is_small(s, q)) {
      const bool pairs = q.r.vals_in != nullptr;
      Group* g = nullptr;
      for (auto& gg : groups)
        if (gg.kt == q.r.kt && gg.desc == q.r.descending && gg.pairs == pairs &&
            gg.reqs.size() < kMaxBatchSegs && gg.keys + q.r.n <= s->cfg.batch_max_keys)
          g = &gg;
      if (!g) {
        groups.push_back(Group{q.r.kt, q.r.descending, pairs, {}, 0});
        g = &groups.back();
      }
      g->keys += q.r.n;
      g->reqs.push_back(std::move(q));
      continue;
    }
    // large: first come first served among large requests
    if (!large_blocked && launch_solo(s, q, pick_stream(s)) == BCF_OK) continue;
    large_blocked = true;
    keep.push_back(std::move(q));
  }
  for (auto& g : groups) {
    if (g.reqs.size() == 1) {
      // nothing to coalesce with: a lone small request runs on its own, which
      // skips the batch's staging copies
      if (launch_solo(s, g.reqs[0], pick_stream(s)) != BCF_OK) keep.push_back(std::move(g.reqs[0]));
      continue;
    }
    if (launch_batch(s, g.reqs, pick_stream(s)) != BCF_OK) {
      for (auto& q : g.reqs) keep.push_back(std::move(q));  // retry on a later step
    }
  }
  // keep arrival order among what is still waiting
  std::stable_sort(keep.begin(), keep.end(),
                   [](const Req& a, const Req& b) { return a.t_submit < b.t_submit; });
  for (auto& q : keep) s->pending.push_back(std::move(q));
}

}  // namespace

extern "C" {

bcf_status bcf_server_create(const bcf_server_config* cfg, bcf_server** out) {
  if (!cfg || !out || !cfg->arena || cfg->arena_bytes < kAlignB || cfg->streams < 1 ||
      cfg->streams > 64 || (reinterpret_cast<uintptr_t>(cfg->arena) & (kAlignB - 1)))
    return BCF_EINVAL;
  bcf_server* s = new (std::nothrow) bcf_server;
  if (!s) return BCF_ENOMEM;
  s->cfg = *cfg;
  if (s->cfg.batch_max_keys == 0) s->cfg.batch_max_keys = 1ull << 22;
  s->arena.init(cfg->arena_bytes);
  const int ns = cfg->mode == BCF_SERVE_PLAIN ? 1 : cfg->streams;
  for (int i = 0; i < ns; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      bcf_server_destroy(s);
      return BCF_ECUDA;
    }
    s->streams.push_back(st);
  }
  if (cudaHostAlloc(reinterpret_cast<void**>(&s->staging), kStagingSlots * kSlotBytes,
                    cudaHostAllocDefault) != cudaSuccess) {
    s->staging = nullptr;
    bcf_server_destroy(s);
    return BCF_ECUDA;
  }
  for (int i = kStagingSlots - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return BCF_OK;
}

double bcf_server_now(const bcf_server* s) { return s ? now_s(s->t0) : 0.0; }

bcf_status bcf_server_submit(bcf_server* s, const bcf_request* r) {
  if (!s || !r) return BCF_EINVAL;
  if (r->op != BCF_OP_SORT && r->op != BCF_OP_MERGE) return BCF_EINVAL;
  if (r->kt < BCF_U32 || r->kt > BCF_I16) return BCF_EINVAL;
  if ((r->vals_in == nullptr) != (r->vals_out == nullptr)) return BCF_EINVAL;
  Req q;
  q.r = *r;
  if (r->op == BCF_OP_MERGE) {
    if (!r->run_offsets || r->k == 0) return BCF_EINVAL;
    q.runs.assign(r->run_offsets, r->run_offsets + r->k + 1);
    for (uint32_t i = 0; i < r->k; ++i)
      if (q.runs[i + 1] < q.runs[i]) return BCF_EINVAL;
    if (q.runs[0] != 0 || q.runs[r->k] != r->n) return BCF_EINVAL;
  }
  // a request that could never fit is refused at once
  const uint64_t solo = solo_bytes(q);
  if (s->cfg.mode == BCF_SERVE_PLAIN || r->n > s->cfg.small_max) {
    if (solo > s->arena.bytes) return BCF_ENOMEM;
  }
  q.t_submit = now_s(s->t0);
  q.runs.shrink_to_fit();
  s->pending.push_back(std::move(q));
  return BCF_OK;
}

bcf_status bcf_server_step(bcf_server* s, int* inflight_out) {
  if (!s) return BCF_EINVAL;
  reap(s);
  if (s->cfg.mode == BCF_SERVE_PLAIN)
    admit_plain(s);
  else
    admit_served(s);
  if (inflight_out) *inflight_out = static_cast<int>(s->inflight.size());
  return BCF_OK;
}

int bcf_server_poll(bcf_server* s, bcf_completion* out, int max) {
  if (!s || !out || max <= 0) return 0;
  const int n = static_cast<int>(s->done.size()) < max ? static_cast<int>(s->done.size()) : max;
  std::memcpy(out, s->done.data(), n * sizeof(bcf_completion));
  s->done.erase(s->done.begin(), s->done.begin() + n);
  return n;
}

bcf_status bcf_server_stats(const bcf_server* s, bcf_server_stats_t* out) {
  if (!s || !out) return BCF_EINVAL;
  out->pending = s->pending.size();
  out->inflight = s->inflight.size();
  out->arena_used = s->arena.used;
  out->arena_peak = s->arena.peak;
  out->launched_units = s->launched_units;
  out->launched_batches = s->launched_batches;
  return BCF_OK;
}

bcf_status bcf_server_drain(bcf_server* s) {
  if (!s) return BCF_EINVAL;
  while (!s->pending.empty() || !s->inflight.empty()) {
    for (auto& st : s->streams) cudaStreamSynchronize(st);
    bcf_server_step(s, nullptr);
  }
  return BCF_OK;
}

bcf_status bcf_server_destroy(bcf_server* s) {
  if (!s) return BCF_EINVAL;
  for (auto& st : s->streams) cudaStreamSynchronize(st);
  for (auto& u : s->inflight) cudaEventDestroy(u.ev);
  for (auto& e : s->events) cudaEventDestroy(e);
  for (auto& st : s->streams) cudaStreamDestroy(st);
  if (s->staging) cudaFreeHost(s->staging);
  delete s;
  return BCF_OK;
}

// ---- the arena allocator on its own (host bookkeeping only, no device memory)

struct bcf_arena {
  Arena a;
};

bcf_status bcf_arena_create(uint64_t bytes, bcf_arena** out) {
  if (!out) return BCF_EINVAL;
  bcf_arena* p = new (std::nothrow) bcf_arena;
  if (!p) return BCF_ENOMEM;
  p->a.init(bytes);
  *out = p;
  return BCF_OK;
}
bcf_status bcf_arena_alloc(bcf_arena* p, uint64_t bytes, uint64_t* offset) {
  if (!p || !offset) return BCF_EINVAL;
  return p->a.alloc(bytes, offset) ? BCF_OK : BCF_ENOMEM;
}
bcf_status bcf_arena_free(bcf_arena* p, uint64_t offset, uint64_t bytes) {
  if (!p) return BCF_EINVAL;
  return p->a.release(offset, bytes) ? BCF_OK : BCF_EINVAL;
}
bcf_status bcf_arena_usage(const bcf_arena* p, uint64_t* used, uint64_t* largest_free) {
  if (!p) return BCF_EINVAL;
  if (used) *used = p->a.used;
  if (largest_free) *largest_free = p->a.largest_free();
  return BCF_OK;
}
bcf_status bcf_arena_destroy(bcf_arena* p) {
  delete p;
  return BCF_OK;
}

}  // extern "C"
