// sv_sample.cu -- measurement: the probability vector and finite-shot draws
// (Sec. 5.3: p_i = x_i^2 + y_i^2 for psi_i = x_i + i y_i, normalised on the
// device; a finite-shot run draws basis indices from it).
//
// Draws use exact integer arithmetic so that they do not depend on the order
// of any floating-point sum (a blocked GPU sum and a sequential one agree bit
// for bit):
//   q_i = floor(p_i 2^61), p_i = x_i^2 + y_i^2 in double with each product
//         and the sum rounded once (no fused multiply-add),
//   Q   = sum_i q_i,
//   t_k = floor(floor(u_k 2^53) Q / 2^53) for the caller's uniform u_k,
//   index_k = the smallest i with q_0 + ... + q_i > t_k.
// The state is cut into chunks of 1024 amplitudes: one pass sums q per chunk,
// one CTA scans the chunk sums, and one warp per shot finds the chunk by
// binary search over the prefix and the index by a warp scan inside it.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "sv_internal.h"

namespace sv {
namespace {

constexpr int kChunkLog = 10;  // amplitudes per chunk: 1024 = 32 lanes x 32

template <typename R>
__device__ __forceinline__ uint64_t q_of(const Cx<R>& a) {
  const double x = (double)a.re, y = (double)a.im;
  const double p = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
  return __double2ull_rz(__dmul_rn(p, 2305843009213693952.0));  // p * 2^61, exact scaling
}

template <typename R>
__device__ __forceinline__ double p_of(const Cx<R>& a) {
  const double x = (double)a.re, y = (double)a.im;
  return __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
}

// q sums per chunk; a warp per chunk.
template <typename R>
__global__ void __launch_bounds__(256) k_chunk_sums(const Cx<R>* __restrict__ psi, uint64_t nchunks, int chunk_log,
                                                    uint64_t* __restrict__ sums) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t c = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += warps) {
    const Cx<R>* a = psi + (c << chunk_log);
    uint64_t s = 0;
    for (int i = lane; i < (1 << chunk_log); i += 32) s += q_of(a[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sums[c] = s;
  }
}

// Exclusive prefix of the chunk sums into pre[0..n], pre[n] = Q (one CTA).
__global__ void __launch_bounds__(1024) k_scan_chunks(const uint64_t* __restrict__ sums, uint64_t n,
                                                      uint64_t* __restrict__ pre) {
  __shared__ uint64_t part[1024];
  const uint64_t per = (n + blockDim.x - 1) / blockDim.x;
  const uint64_t b = threadIdx.x * per, e = b + per < n ? b + per : n;
  uint64_t s = 0;
  for (uint64_t i = b; i < e; i++) s += sums[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {  // inclusive scan of the segment sums
    const uint64_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint64_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (uint64_t i = b; i < e; i++) {
    pre[i] = run;
    run += sums[i];
  }
  if (threadIdx.x == blockDim.x - 1) pre[n] = part[blockDim.x - 1];
}

// One warp per shot.
template <typename R>
__global__ void __launch_bounds__(256) k_draw(const Cx<R>* __restrict__ psi, const uint64_t* __restrict__ pre,
                                              uint64_t nchunks, int chunk_log, const double* __restrict__ u,
                                              uint64_t nshots, uint64_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t Q = pre[nchunks];
  for (uint64_t k = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); k < nshots; k += warps) {
    const uint64_t m = __double2ull_rz(__dmul_rn(u[k], 9007199254740992.0));  // floor(u 2^53)
    const uint64_t lo = m * Q, hi = __umul64hi(m, Q);
    const uint64_t t = (hi << 11) | (lo >> 53);  // floor(m Q / 2^53) < Q
    // the chunk c with pre[c] <= t < pre[c + 1]
    uint64_t a = 0, b = nchunks - 1;
    while (a < b) {
      const uint64_t mid = (a + b + 1) >> 1;
      if (pre[mid] <= t)
        a = mid;
      else
        b = mid - 1;
    }
    const uint64_t r = t - pre[a];
    // lane segments of 2^(chunk_log - 5) amplitudes, scanned across the warp
    const int seg_log = chunk_log - 5;
    const Cx<R>* base = psi + (a << chunk_log) + ((uint64_t)lane << seg_log);
    uint64_t s = 0;
    for (int i = 0; i < (1 << seg_log); i++) s += q_of(base[i]);
    uint64_t inc = s;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    const uint64_t exc = inc - s;
    const unsigned owner = __ballot_sync(0xffffffffu, exc <= r && r < inc);
    if (owner) {
      const int L = __ffs(owner) - 1;
      if (lane == L) {
        uint64_t run = exc;
        int i = 0;
        for (; i < (1 << seg_log) - 1; i++) {
          run += q_of(base[i]);
          if (run > r) break;
        }
        out[k] = (a << chunk_log) + ((uint64_t)lane << seg_log) + (uint64_t)i;
      }
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_probs(const Cx<R>* __restrict__ psi, uint64_t N, double* __restrict__ p) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = p_of(psi[i]);
}

__global__ void __launch_bounds__(256) k_scale(double* __restrict__ p, uint64_t N, const double* __restrict__ tot) {
  const double s = *tot;
  if (!(s > 0.0)) return;
  const double inv = 1.0 / s;  // one FP64 multiply per entry (FP64 division is slow on GB300)
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] *= inv;
}

// Sum of p in double over a warp per 1024 entries, then one CTA (fixed order).
__global__ void __launch_bounds__(256) k_psum(const double* __restrict__ p, uint64_t nchunks, int chunk_log,
                                              double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t c = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += warps) {
    double s = 0.0;
    for (int i = lane; i < (1 << chunk_log); i += 32) s += p[(c << chunk_log) + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[c] = s;
  }
}

__global__ void __launch_bounds__(1024) k_psum_final(const double* __restrict__ part, uint64_t n,
                                                     double* __restrict__ tot) {
  __shared__ double red[1024];
  double s = 0.0;
  for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *tot = red[0];
}

unsigned grid_for(uint64_t work_items, int per_block) {
  uint64_t g = (work_items + per_block - 1) / per_block;
  const uint64_t cap = (uint64_t)device_sm_count() * 8;
  if (g > cap) g = cap;
  return (unsigned)(g ? g : 1);
}

template <typename R>
void probabilities(const Cx<R>* psi, int n, double* p, bool normalise, cudaStream_t s) {
  const uint64_t N = 1ull << n;
  k_probs<R><<<grid_for(N, 256), 256, 0, s>>>(psi, N, p);
  cuda_check(cudaGetLastError(), "probabilities");
  if (!normalise) return;
  const int cl = n < kChunkLog ? n : kChunkLog;
  const uint64_t nch = N >> cl;
  double* part = (double*)scratch_buffer(s, "prob_partials", sizeof(double) * (nch + 1));
  k_psum<<<grid_for(nch, 8), 256, 0, s>>>(p, nch, cl, part);
  k_psum_final<<<1, 1024, 0, s>>>(part, nch, part + nch);
  k_scale<<<grid_for(N, 256), 256, 0, s>>>(p, N, part + nch);
  cuda_check(cudaGetLastError(), "probabilities (normalise)");
}

template <typename R>
void sample(const Cx<R>* psi, int n, const double* u_host, size_t nshots, uint64_t* out, bool out_on_device,
            cudaStream_t s) {
  const int cl = n < kChunkLog ? n : kChunkLog;
  if (cl < 5) fail(SV_ERR_UNSUPPORTED, "sampling needs n_qubits >= 5 (32-amplitude lane segments)");
  const uint64_t N = 1ull << n, nch = N >> cl;
  uint64_t* sums = (uint64_t*)scratch_buffer(s, "sample_sums", sizeof(uint64_t) * (2 * nch + 1));
  uint64_t* pre = sums + nch;
  double* du = (double*)scratch_buffer(s, "sample_u", sizeof(double) * nshots);
  uint64_t* dout = out_on_device ? out : (uint64_t*)scratch_buffer(s, "sample_out", sizeof(uint64_t) * nshots);
  cuda_check(cudaMemcpyAsync(du, u_host, sizeof(double) * nshots, cudaMemcpyHostToDevice, s), "uniforms upload");
  k_chunk_sums<R><<<grid_for(nch, 8), 256, 0, s>>>(psi, nch, cl, sums);
  k_scan_chunks<<<1, 1024, 0, s>>>(sums, nch, pre);
  uint64_t Q = 0;
  cuda_check(cudaMemcpyAsync(&Q, pre + nch, sizeof(Q), cudaMemcpyDeviceToHost, s), "total read");
  cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (Q == 0) fail(SV_ERR_INVALID, "the state has no probability mass above 2^-61");
  k_draw<R><<<grid_for(nshots, 8), 256, 0, s>>>(psi, pre, nch, cl, du, nshots, dout);
  cuda_check(cudaGetLastError(), "draw");
  if (!out_on_device) {
    cuda_check(cudaMemcpyAsync(out, dout, sizeof(uint64_t) * nshots, cudaMemcpyDeviceToHost, s), "result read");
    cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  }
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_probabilities(const void* state, int n_qubits, sv_dtype dtype, double* out, int normalise,
                                      void* stream) {
  return guarded([&] {
    if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_INVALID, "unknown dtype");
    if (n_qubits < 1 || n_qubits > SV_MAX_QUBITS) fail(SV_ERR_INVALID, "n_qubits must be in 1..34");
    const size_t amp = dtype == SV_C64 ? 8 : 16;
    check_device_buffer(state, amp << n_qubits, "state");
    check_device_buffer(out, sizeof(double) << n_qubits, "out");
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SV_C64)
      probabilities<float>((const Cx<float>*)state, n_qubits, out, normalise != 0, s);
    else
      probabilities<double>((const Cx<double>*)state, n_qubits, out, normalise != 0, s);
  });
}

extern "C" sv_status sv_sample(const void* state, int n_qubits, sv_dtype dtype, const double* uniforms,
                               size_t n_shots, uint64_t* out, int out_on_device, void* stream) {
  return guarded([&] {
    if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_INVALID, "unknown dtype");
    if (n_qubits < 5 || n_qubits > SV_MAX_QUBITS) fail(SV_ERR_INVALID, "n_qubits must be in 5..34");
    if (n_shots == 0) return;
    if (!uniforms || !out) fail(SV_ERR_INVALID, "uniforms or out is NULL");
    for (size_t k = 0; k < n_shots; k++)
      if (!(uniforms[k] >= 0.0 && uniforms[k] < 1.0)) fail(SV_ERR_INVALID, "uniforms must lie in [0, 1)");
    const size_t amp = dtype == SV_C64 ? 8 : 16;
    check_device_buffer(state, amp << n_qubits, "state");
    if (out_on_device) check_device_buffer(out, sizeof(uint64_t) * n_shots, "out");
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SV_C64)
      sample<float>((const Cx<float>*)state, n_qubits, uniforms, n_shots, out, out_on_device != 0, s);
    else
      sample<double>((const Cx<double>*)state, n_qubits, uniforms, n_shots, out, out_on_device != 0, s);
  });
}
