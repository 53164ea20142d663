// bcf_segmented_u32.cu -- the persistent segmented sort instantiated for uint32_t keys
// without payloads, and the worker's wait self-test.
#include "bcf_segmented.cuh"

namespace bcf {

template cudaError_t launch_segmented_kp<uint32_t, false>(int, const SegArgs&, cudaStream_t);

// Failure-path self-test of the worker's wait for a queue slot: the queue
// announces one work item (total = 1) whose slot is never published (its
// ready bit stays clear), so the one worker CTA that takes it waits, bounded
// by wait_ns, records kErrQueueTimeout and exits without touching any data.
static __global__ void seg_selftest_init(SegCtl* ctl, SegWork* queue) {
  ctl->head = 0;
  ctl->reserve = 1;
  ctl->total = 1;
  ctl->n_tiny = 0;
  queue[0].meta = 0;  // announced, never published
  queue[0].seg = 0;
  queue[0].arg = 0;
}

cudaError_t launch_segmented_wait_selftest(void* ws, uint64_t wait_ns, uint32_t* err,
                                           cudaStream_t s) {
  constexpr int E = 16, NT = 256;
  SegArgs a{};
  char* w = static_cast<char*>(ws);
  a.ctl = reinterpret_cast<SegCtl*>(w);
  a.queue = reinterpret_cast<SegWork*>(w + 256);
  a.capacity = 1;
  a.off = reinterpret_cast<const uint64_t*>(w + 384);  // never read: no slot is ready
  a.nseg = 0;
  a.n = 0;
  a.err = err;
  a.wait_ns = wait_ns;
  seg_selftest_init<<<1, 1, 0, s>>>(a.ctl, a.queue);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  auto kern = seg_kernel<uint32_t, false, E, NT, false>();
  const size_t smem = Geo<E, NT>::kPlane * sizeof(uint32_t);
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem))) != cudaSuccess)
    return e;
  kern<<<1, NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace bcf
