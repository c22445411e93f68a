// sv_noalloc.cu -- sv_expect_z_all_noalloc: the per-qubit <Z> read-out without
// any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a serving process that
// has handed all device memory to its own pool and must not grow, code that
// must not stall other streams (cudaMalloc and cudaFree can synchronize the
// device), or a host framework that owns every device byte through its own
// allocator.  For them this entry point runs the same two kernels as
// sv_expect_z_all, but its per-block partial sums live in a fixed array in the
// library's own device memory (below) instead of library-allocated scratch.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoallocRows x (SV_MAX_QUBITS + 1) doubles = 280 KiB)
// until the process exits.  In host code its name is only a host-side stand-in,
// not a device address, so the address is taken with cudaGetSymbolAddress once
// per device, with that device current, the first time this entry point runs
// there; that first call should come before any stream capture.  Every call
// shares the array: calls whose kernels overlap on the GPU (for example on two
// streams at once) race on it and may return wrong values.  Each call fully
// rewrites the rows it reads, so nothing needs clearing between calls.
#include <cuda_runtime.h>

#include <mutex>

#include "sv_internal.h"

namespace sv {
namespace {

constexpr int kNoallocRows = 1024;  // per-block partial rows (a grid of up to 1024 blocks)
constexpr size_t kNoallocDoubles = (size_t)kNoallocRows * (SV_MAX_QUBITS + 1);

static __device__ __align__(256) double g_noalloc_partials[kNoallocDoubles];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {nullptr};

// Device address of g_noalloc_partials on the current device (set up once).
double* noalloc_scratch() {
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64) fail(SV_ERR_INVALID, "device index beyond 63");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      fail(SV_ERR_CUDA, std::string("cudaGetSymbolAddress of the fixed scratch failed: ") + cudaGetErrorString(e));
    }
    g_noalloc_ptr[dev] = (double*)p;
  }
  return g_noalloc_ptr[dev];
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_expect_z_all_noalloc(const void* state, int n_qubits, sv_dtype dtype, double* out,
                                             void* stream) {
  return guarded([&] {
    if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_INVALID, "unknown dtype");
    if (n_qubits < 1 || n_qubits > SV_MAX_QUBITS)
      fail(SV_ERR_INVALID, "n_qubits must be in 1..34: the fixed scratch holds rows of at most 35 doubles");
    if (!out) fail(SV_ERR_INVALID, "out is NULL");
    const size_t amp = dtype == SV_C64 ? 8 : 16;
    check_device_buffer(state, amp << n_qubits, "state");
    check_device_buffer(out, sizeof(double) * (n_qubits + 1), "out");
    double* scratch = noalloc_scratch();
    if (expect_z_all_scratch_doubles(n_qubits) > kNoallocDoubles)
      fail(SV_ERR_INVALID, "this GPU needs more partial rows than the fixed scratch holds (1024)");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = dtype == SV_C64
                        ? launch_expect_z_all<float>((const Cx<float>*)state, n_qubits, scratch, kNoallocDoubles, out, s)
                        : launch_expect_z_all<double>((const Cx<double>*)state, n_qubits, scratch, kNoallocDoubles,
                                                      out, s);
    cuda_check(e, "expect_z_all launch");
  });
}
