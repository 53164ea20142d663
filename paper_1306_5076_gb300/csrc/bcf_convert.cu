// bcf_convert.cu -- element conversions used to build the 16-bit key types
// and the wide payloads out of the 32-bit sort (the extension types of the
// library; the paper sorts 32-bit unsigned keys only, Sec. 4).
//
//   widen16   u16 -> u32 (zero extension) or i16 -> i32 (sign extension):
//             order-preserving, so sorting the widened keys sorts the keys;
//   narrow16  the inverse (the low 16 bits);
//   iota      v[i] = i, the row index carried through a pairs sort;
//   gather    out[i] = in[idx[i]] for rows of `row_bytes` bytes (a multiple
//             of 4): the payloads of a sort by key, permuted by the sorted
//             row indices (one thread per row, widest aligned vectors).
#include <cuda_runtime.h>

#include "bcf_internal.h"

namespace bcf {

namespace {

constexpr int kThreads = 256;

__global__ void widen16_kernel(uint32_t* out, const uint16_t* in, uint64_t n, int sign) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint16_t x = in[i];
    out[i] = sign ? static_cast<uint32_t>(static_cast<int32_t>(static_cast<int16_t>(x)))
                  : static_cast<uint32_t>(x);
  }
}

__global__ void narrow16_kernel(uint16_t* out, const uint32_t* in, uint64_t n) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    out[i] = static_cast<uint16_t>(in[i]);
}

__global__ void iota_kernel(uint32_t* v, uint64_t n) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    v[i] = static_cast<uint32_t>(i);
}

// One thread per row: the row's words are copied as vectors of V words
// (16-, 8- or 4-byte accesses), reading a scattered row, writing rows in order.
template <typename Vec>
__global__ void gather_kernel(Vec* out, const Vec* in, const uint32_t* idx, uint64_t n,
                              uint32_t vecs) {
  for (uint64_t r = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const Vec* src = in + static_cast<uint64_t>(idx[r]) * vecs;
    Vec* dst = out + r * vecs;
    for (uint32_t c = 0; c < vecs; ++c) dst[c] = src[c];
  }
}

unsigned grid_for(uint64_t work) {
  const uint64_t blocks = (work + kThreads - 1) / kThreads;
  return static_cast<unsigned>(blocks < 152ull * 32 ? (blocks ? blocks : 1) : 152ull * 32);
}

}  // namespace

cudaError_t launch_widen16(uint32_t* out, const uint16_t* in, uint64_t n, bool sign,
                           cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  widen16_kernel<<<grid_for(n), kThreads, 0, s>>>(out, in, n, sign ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t launch_narrow16(uint16_t* out, const uint32_t* in, uint64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  narrow16_kernel<<<grid_for(n), kThreads, 0, s>>>(out, in, n);
  return cudaGetLastError();
}
cudaError_t launch_iota(uint32_t* v, uint64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  iota_kernel<<<grid_for(n), kThreads, 0, s>>>(v, n);
  return cudaGetLastError();
}
cudaError_t launch_gather(void* out, const void* in, const uint32_t* idx, uint64_t n,
                          uint32_t row_bytes, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uintptr_t align = reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(in);
  if (row_bytes % 16 == 0 && align % 16 == 0)
    gather_kernel<uint4><<<grid_for(n), kThreads, 0, s>>>(
        static_cast<uint4*>(out), static_cast<const uint4*>(in), idx, n, row_bytes / 16);
  else if (row_bytes % 8 == 0 && align % 8 == 0)
    gather_kernel<uint2><<<grid_for(n), kThreads, 0, s>>>(
        static_cast<uint2*>(out), static_cast<const uint2*>(in), idx, n, row_bytes / 8);
  else
    gather_kernel<uint32_t><<<grid_for(n), kThreads, 0, s>>>(
        static_cast<uint32_t*>(out), static_cast<const uint32_t*>(in), idx, n, row_bytes / 4);
  return cudaGetLastError();
}

}  // namespace bcf
