// sv_hostcopy.h -- state copies between device memory and host memory
// (sv_hostcopy.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace sv {

// True when `host` is 16-byte aligned page-locked memory mapped into the
// current device at the same address (checked at both ends of the range) and
// bytes is a whole number of 16-byte vectors: such copies run as a kernel.
bool host_copy_by_sm(const void* host, size_t bytes);

// Copies `bytes` between device memory and host memory on `stream`
// (to_host: device src -> host dst; else host src -> device dst), by a kernel
// of SM loads and stores when host_copy_by_sm holds for the host side and the
// device side is 16-byte aligned, else by cudaMemcpyAsync.  Asynchronous; the
// result is the launch's or the copy's error.
cudaError_t copy_state_host(void* dst, const void* src, size_t bytes, bool to_host, cudaStream_t stream);

}  // namespace sv
