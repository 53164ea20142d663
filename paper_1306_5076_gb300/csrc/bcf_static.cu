// bcf_static.cu -- bcf_sort_keys_static: the key sort with its scratch memory
// in a file-scope device array instead of a caller-provided workspace.
//
// Who needs it: callers that cannot call cudaMalloc at all -- for example a
// plugin or kernel-hosting framework that owns every device allocation and
// hands a plugin only its input and output buffers, a process whose device
// memory is carved up by an external pool it must not go around, or a
// latency-critical loop that must never hit cudaMalloc's implicit
// device-wide synchronisation.  Such callers pass inputs and outputs only;
// the ping-pong buffer and split array of the merge passes live in
// g_static_workspace below, reserved when the library is loaded on a GPU.
//
// Costs and rules:
//  - every GPU that loads this library holds kStaticBytes (about 8.1 MiB) of
//    device memory until the process exits;
//  - at most BCF_STATIC_MAX_KEYS keys per call;
//  - every call shares the one array: calls whose GPU work overlaps (two
//    streams, or two host threads) race and corrupt each other's results;
//  - nothing in the array has to start at zero (every word is written before
//    it is read), so calls need not clear it; it keeps the last call's data;
//  - the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current.
#include <cuda_runtime.h>

#include <mutex>

#include "bcf_internal.h"
#include "bcfsort.h"

namespace {

// The sort's workspace for BCF_STATIC_MAX_KEYS keys of the widest type (u64),
// keys only, by the same formula bcf_workspace_bytes uses (a workspace for
// fewer or narrower keys is never larger).
constexpr size_t kMaxKeys = BCF_STATIC_MAX_KEYS;
constexpr size_t kStaticBytes = bcf::ws_layout(kMaxKeys, 0, 8, false).total;
static_assert(kStaticBytes < (size_t(9) << 20), "static scratch larger than documented");

static __device__ __align__(256) unsigned char g_static_workspace[kStaticBytes];

// Device address of g_static_workspace on the current device (its host-side
// name is only a stand-in; kernels must be given this address).
void* static_workspace() {
  static std::mutex mu;
  static void* addr[64] = {};
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_workspace) != cudaSuccess) return nullptr;
    addr[dev] = p;
  }
  return addr[dev];
}

}  // namespace

extern "C" bcf_status bcf_sort_keys_static(void* keys_out, const void* keys_in, uint64_t n,
                                           bcf_dtype kt, const bcf_opts* opts,
                                           cudaStream_t stream) {
  if (n > kMaxKeys) return BCF_EUNSUPPORTED;
  // 16-bit keys need widened copies the static array has no room for
  if (kt == BCF_U16 || kt == BCF_I16) return BCF_EUNSUPPORTED;
  // the static array is sized for the merge path: pivot buckets and the
  // automatic choice take it too; any other algorithm value reaches
  // bcf_sort_keys and is rejected there
  bcf_opts o{};
  if (opts) o = *opts;
  if (o.algorithm == BCF_ALGO_PIVOT_BUCKETS || o.algorithm == BCF_ALGO_AUTO)
    o.algorithm = BCF_ALGO_MERGE;
  if (n == 0) return bcf_sort_keys(keys_out, keys_in, 0, kt, &o, nullptr, 0, stream);
  void* ws = static_workspace();
  if (!ws) return BCF_ECUDA;
  return bcf_sort_keys(keys_out, keys_in, n, kt, &o, ws, kStaticBytes, stream);
}
