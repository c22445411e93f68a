// sv_hostcopy.cu -- state copies between device memory and page-locked host
// memory by SM loads and stores (the explicit exit to and entry from the host,
// Sec. 5.1), used by sv_run_host, sv_set_state and sv_get_state.
//
// Page-locked host memory that the runtime maps into the device's address
// space (cudaHostAlloc / cudaMallocHost buffers under unified addressing, and
// so every pinned torch tensor) can be written and read by a kernel over the
// CPU-GPU link.  On GB300 with its Grace host both routes top out near
// 193 GB/s device-to-host when warm, but a copy-engine transfer of a
// multi-gigabyte state that starts after the link has idled (behind ~100 ms of
// kernels, or 1 s of nothing) was measured at 17-30 GB/s, and host CPU
// activity did not change that, while SM stores into the same buffer held
// 120-190 GB/s.  A state download follows the circuit's kernels, so it is
// always in that position.  Host memory that is not mapped (pageable memory,
// or a pinned range the runtime reports no device address for) keeps
// cudaMemcpyAsync, as do sizes that are not whole 16-byte vectors.
#include <cuda_runtime.h>

#include <cstdint>

#include "sv_hostcopy.h"
#include "sv_internal.h"

namespace sv {
namespace {

constexpr int kCopyThreads = 256;
constexpr int kCopyUnroll = 4;  // 16-byte vectors in flight per thread per step

// dst[i] = src[i] for i < n16 (16-byte vectors).  Each thread moves kCopyUnroll
// vectors a step, blockDim apart so that a warp's accesses stay contiguous; the
// last, partial step checks every index.
__global__ void __launch_bounds__(kCopyThreads) k_copy16(uint4* __restrict__ dst, const uint4* __restrict__ src,
                                                         size_t n16) {
  const size_t bd = blockDim.x;
  const size_t stride = (size_t)gridDim.x * bd * kCopyUnroll;
  size_t base = (size_t)blockIdx.x * bd * kCopyUnroll + threadIdx.x;
  for (; base + (kCopyUnroll - 1) * bd < n16; base += stride) {
    uint4 v[kCopyUnroll];
#pragma unroll
    for (int u = 0; u < kCopyUnroll; u++) v[u] = src[base + u * bd];
#pragma unroll
    for (int u = 0; u < kCopyUnroll; u++) dst[base + u * bd] = v[u];
  }
#pragma unroll
  for (int u = 0; u < kCopyUnroll; u++)
    if (base + u * bd < n16) dst[base + u * bd] = src[base + u * bd];
}

// True when the host range [p, p + bytes) starts and ends in page-locked
// memory that the current device reaches at the same address.
bool mapped_host_range(const void* p, size_t bytes) {
  if (bytes == 0) return false;
  const char* c = static_cast<const char*>(p);
  for (const char* q : {c, c + bytes - 1}) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (at.type != cudaMemoryTypeHost || at.devicePointer != static_cast<const void*>(q)) return false;
  }
  return true;
}

}  // namespace

bool host_copy_by_sm(const void* host, size_t bytes) {
  return bytes > 0 && bytes % 16 == 0 && (uintptr_t)host % 16 == 0 && mapped_host_range(host, bytes);
}

cudaError_t copy_state_host(void* dst, const void* src, size_t bytes, bool to_host, cudaStream_t stream) {
  const void* host = to_host ? static_cast<const void*>(dst) : src;
  if (!host_copy_by_sm(host, bytes) || (uintptr_t)(to_host ? src : dst) % 16 != 0)
    return cudaMemcpyAsync(dst, src, bytes, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice, stream);
  const size_t n16 = bytes / 16;
  const size_t per_block = (size_t)kCopyThreads * kCopyUnroll;
  size_t grid = (n16 + per_block - 1) / per_block;
  const size_t cap = (size_t)device_sm_count() * 8;  // 2048 threads per SM resident
  if (grid > cap) grid = cap;
  Prof p(stream, to_host ? "host_store" : "host_load", (double)bytes);
  k_copy16<<<(unsigned)grid, kCopyThreads, 0, stream>>>(static_cast<uint4*>(dst), static_cast<const uint4*>(src),
                                                        n16);
  p.done();
  return cudaGetLastError();
}

}  // namespace sv
