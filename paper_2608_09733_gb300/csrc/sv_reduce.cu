// sv_reduce.cu -- read-only expectation reductions for sm_103a.
//
// <Z_q> for every qubit in one pass (Sec. 5.3 probabilities p_b = x_b^2 + y_b^2,
// Sec. 4.4 Pauli path): <Z_q> = T - 2 S_q with T = sum_b p_b and S_q the sum
// over the amplitudes whose bit q is set.  A warp owns a chunk of 32 x 32
// 16-byte vectors; inside a chunk the low index bits are the vector element,
// the lane and the iteration, so S_q for those bits is accumulated with
// compile-time-known adds and a warp butterfly; bits above the chunk are the
// same for the whole chunk.
//
// General Pauli terms (Sec. 4.4): <psi|P|psi> = i^{nY} sum_b (-1)^{popc(b&z)}
// conj(psi_{b^x}) psi_b.  For x != 0 the sum is taken over half the indices
// (bit h = top bit of x clear) and doubled: the partner's term is the complex
// conjugate of this one, so <P> = 2 Re[i^{nY} sum_half ...].  Terms that share
// an x mask share one pass.
//
// Precision (complex64): each thread sums p in float over a short run (64
// amplitudes); the warp adds its 32 runs in float (a chunk of 2048
// amplitudes: relative error below 70 float roundings, 4e-6, of the chunk's
// sum) and the chunk sums go into double, as do the block and grid
// reductions.  (Warp sums in double took most of the kernel's time: the FP64
// pipe of this part runs a warp-wide add in about 16 cycles.)  complex128
// accumulates in double throughout.
// The grid writes one partial per block and a one-block kernel adds them in a
// fixed order, so results are identical run to run.
#include <cuda_runtime.h>

#include "sv_internal.h"

namespace sv {

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedWarps = kRedThreads / 32;
constexpr int kJ = 32;          // vectors per lane per chunk
constexpr int kMaxTermsPerPass = 16;

int red_grid() { return device_sm_count() * 4; }

template <typename R>
struct Acc;  // accumulation type for short runs
template <>
struct Acc<float> {
  using T = float;
};
template <>
struct Acc<double> {
  using T = double;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------ <Z_q> for all q

// A = amplitudes per 16-byte vector (2 for complex64, 1 for complex128).
// Chunk = 32 lanes x kJ vectors x A amplitudes; chunk bits C = log2(1024 A).
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_expect_z_all(const Cx<R>* __restrict__ state, int n,
                                                            double* __restrict__ partials) {
  constexpr int A = 16 / sizeof(Cx<R>);
  constexpr int EB = (A == 2) ? 1 : 0;  // index bits taken by the vector element
  constexpr int C = EB + 5 + 5;         // chunk bits
  using T = typename Acc<R>::T;
  __shared__ double red[kRedWarps][SV_MAX_QUBITS + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t nchunks = 1ull << (n - C);
  const uint64_t gwarp = (uint64_t)blockIdx.x * kRedWarps + warp;
  const uint64_t nwarps = (uint64_t)gridDim.x * kRedWarps;
  double accq0 = 0.0, accq1 = 0.0, acct = 0.0;  // qubits lane and lane + 32; total
  for (uint64_t ch = gwarp; ch < nchunks; ch += nwarps) {
    const uint4* src = reinterpret_cast<const uint4*>(state + (ch << C));
    T tot = 0, e1 = 0, jb0 = 0, jb1 = 0, jb2 = 0, jb3 = 0, jb4 = 0;
#pragma unroll
    for (int j = 0; j < kJ; j++) {
      uint4 w = __ldg(src + j * 32 + lane);
      T p;
      if constexpr (A == 2) {
        float2 a = *reinterpret_cast<float2*>(&w.x), b = *reinterpret_cast<float2*>(&w.z);
        T p0 = fmaf(a.x, a.x, a.y * a.y), p1 = fmaf(b.x, b.x, b.y * b.y);
        e1 += p1;
        p = p0 + p1;
      } else {
        double2 a = *reinterpret_cast<double2*>(&w);
        p = fma(a.x, a.x, a.y * a.y);
      }
      tot += p;
      if (j & 1) jb0 += p;
      if (j & 2) jb1 += p;
      if (j & 4) jb2 += p;
      if (j & 8) jb3 += p;
      if (j & 16) jb4 += p;
    }
    // reduce the lanes' runs across the warp (in the run's precision), then
    // into double
    const double t = (double)warp_sum(tot);
    const double v_e1 = EB ? (double)warp_sum(e1) : 0.0;
    const double v_j[5] = {(double)warp_sum(jb0), (double)warp_sum(jb1), (double)warp_sum(jb2),
                           (double)warp_sum(jb3), (double)warp_sum(jb4)};
    double v_l[5];
#pragma unroll
    for (int b = 0; b < 5; b++) v_l[b] = (double)warp_sum(((lane >> b) & 1) ? tot : T(0));
    // lane q picks S_q for its qubits q = lane and lane + 32
#pragma unroll
    for (int rep = 0; rep < 2; rep++) {
      const int q = lane + 32 * rep;
      if (q >= n) continue;
      double sq;
      if (q >= C) {
        sq = ((ch >> (q - C)) & 1ull) ? t : 0.0;
      } else if (EB && q == 0) {
        sq = v_e1;
      } else if (q < EB + 5) {
        int b = q - EB;
        sq = b == 0 ? v_l[0] : b == 1 ? v_l[1] : b == 2 ? v_l[2] : b == 3 ? v_l[3] : v_l[4];
      } else {
        int b = q - EB - 5;
        sq = b == 0 ? v_j[0] : b == 1 ? v_j[1] : b == 2 ? v_j[2] : b == 3 ? v_j[3] : v_j[4];
      }
      if (rep == 0) accq0 += sq; else accq1 += sq;
    }
    acct += t;
  }
  if (lane < n) red[warp][lane] = accq0;
  if (lane + 32 < n) red[warp][lane + 32] = accq1;
  if (lane == 0) red[warp][n] = acct;
  __syncthreads();
  for (int q = threadIdx.x; q <= n; q += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kRedWarps; w++) s += red[w][q];
    partials[(size_t)blockIdx.x * (n + 1) + q] = s;
  }
}

// Small states (n below one warp chunk): one thread per amplitude, direct.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_expect_z_small(const Cx<R>* __restrict__ state, int n,
                                                              double* __restrict__ partials) {
  __shared__ double red[SV_MAX_QUBITS + 1];
  if (blockIdx.x != 0) return;
  for (int q = threadIdx.x; q <= n; q += blockDim.x) {
    double s = 0.0;
    for (uint32_t b = 0; b < (1u << n); b++) {
      Cx<R> a = state[b];
      double p = (double)a.re * a.re + (double)a.im * a.im;
      if (q == n || ((b >> q) & 1u)) s += p;
    }
    red[q] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q <= n; q += blockDim.x) partials[q] = red[q];
}

__global__ void k_finish_z_all(const double* __restrict__ partials, int nblocks, int n, double* __restrict__ out) {
  __shared__ double s[SV_MAX_QUBITS + 1];
  for (int q = threadIdx.x; q <= n; q += blockDim.x) {
    double a = 0.0;
    for (int b = 0; b < nblocks; b++) a += partials[(size_t)b * (n + 1) + q];
    s[q] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double T = s[n];
    double sum = 0.0;
    for (int q = 0; q < n; q++) {
      double z = T - 2.0 * s[q];
      out[q] = z;
      sum += z;
    }
    out[n] = sum;
  }
}

// ------------------------------------------------------------ Pauli terms

struct TermPass {
  uint64_t x;
  int h;        // top bit of x, or -1 when x == 0
  int nt;
  uint64_t z[kMaxTermsPerPass];
};

template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_expect_terms(const Cx<R>* __restrict__ state, int n, TermPass tp,
                                                            double* __restrict__ partials) {
  using T = typename Acc<R>::T;
  __shared__ double red[kRedWarps][kMaxTermsPerPass][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t count = tp.h >= 0 ? (1ull << (n - 1)) : (1ull << n);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double are[kMaxTermsPerPass], aim[kMaxTermsPerPass];
#pragma unroll
  for (int j = 0; j < kMaxTermsPerPass; j++) are[j] = aim[j] = 0.0;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  while (i < count) {
    T rre[kMaxTermsPerPass], rim[kMaxTermsPerPass];
#pragma unroll
    for (int j = 0; j < kMaxTermsPerPass; j++) rre[j] = rim[j] = 0;
    // a short run in the run precision, then fold into double
    for (int r = 0; r < 64 && i < count; r++, i += stride) {
      uint64_t b = tp.h >= 0 ? ((i >> tp.h) << (tp.h + 1)) | (i & ((1ull << tp.h) - 1ull)) : i;
      Cx<R> a = state[b];
      T vre, vim;
      if (tp.h >= 0) {
        Cx<R> c = state[b ^ tp.x];  // conj(c) * a
        vre = (T)c.re * (T)a.re + (T)c.im * (T)a.im;
        vim = (T)c.re * (T)a.im - (T)c.im * (T)a.re;
      } else {
        vre = (T)a.re * (T)a.re + (T)a.im * (T)a.im;
        vim = 0;
      }
#pragma unroll
      for (int j = 0; j < kMaxTermsPerPass; j++) {
        if (j < tp.nt) {
          T sg = (__popcll(b & tp.z[j]) & 1) ? T(-1) : T(1);
          rre[j] = fma(sg, vre, rre[j]);
          rim[j] = fma(sg, vim, rim[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxTermsPerPass; j++) {
      are[j] += (double)rre[j];
      aim[j] += (double)rim[j];
    }
  }
#pragma unroll
  for (int j = 0; j < kMaxTermsPerPass; j++) {
    double a = warp_sum(are[j]), b = warp_sum(aim[j]);
    if (lane == 0 && j < tp.nt) {
      red[warp][j][0] = a;
      red[warp][j][1] = b;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < tp.nt; j += blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kRedWarps; w++) {
      a += red[w][j][0];
      b += red[w][j][1];
    }
    partials[((size_t)blockIdx.x * kMaxTermsPerPass + j) * 2] = a;
    partials[((size_t)blockIdx.x * kMaxTermsPerPass + j) * 2 + 1] = b;
  }
}

struct TermOut {
  int nt;
  int dst[kMaxTermsPerPass];  // output index of each term of the pass
  int ny[kMaxTermsPerPass];   // number of Y letters
};

__global__ void k_finish_terms(const double* __restrict__ partials, int nblocks, int paired, TermOut to,
                               double* __restrict__ out) {
  int j = threadIdx.x;
  if (j >= to.nt) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nblocks; k++) {
    a += partials[((size_t)k * kMaxTermsPerPass + j) * 2];
    b += partials[((size_t)k * kMaxTermsPerPass + j) * 2 + 1];
  }
  // Re[i^{nY} (a + i b)]
  double re;
  switch (to.ny[j] & 3) {
    case 0: re = a; break;
    case 1: re = -b; break;
    case 2: re = -a; break;
    default: re = b; break;
  }
  out[to.dst[j]] = paired ? 2.0 * re : re;
}

}  // namespace

// Sized for the largest state whatever n is, so the per-stream scratch never
// regrows: regrowing frees the old buffer, and cudaFree synchronizes the whole
// device (it would wait for a resident serving kernel).
size_t expect_z_all_scratch_doubles(int n) {
  (void)n;
  return (size_t)red_grid() * (SV_MAX_QUBITS + 1);
}
size_t expect_terms_scratch_doubles(int n, int n_terms) {
  (void)n;
  (void)n_terms;
  return (size_t)red_grid() * kMaxTermsPerPass * 2;
}

template <typename R>
cudaError_t launch_expect_z_all(const Cx<R>* state, int n, double* scratch, size_t scratch_doubles, double* out,
                                cudaStream_t stream) {
  constexpr int A = 16 / sizeof(Cx<R>);
  constexpr int C = (A == 2 ? 1 : 0) + 10;
  int grid;
  if (n < C) {
    grid = 1;
    k_expect_z_small<R><<<1, kRedThreads, 0, stream>>>(state, n, scratch);
  } else {
    uint64_t chunks = 1ull << (n - C);
    uint64_t g = (chunks + kRedWarps - 1) / kRedWarps;
    grid = (int)(g < (uint64_t)red_grid() ? g : (uint64_t)red_grid());
    if ((size_t)grid * (n + 1) > scratch_doubles) return cudaErrorInvalidValue;
    k_expect_z_all<R><<<grid, kRedThreads, 0, stream>>>(state, n, scratch);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_finish_z_all<<<1, 64, 0, stream>>>(scratch, grid, n, out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_expect_terms(const Cx<R>* state, int n, const sv_pauli_term* terms, int n_terms, double* scratch,
                                size_t scratch_doubles, double* out, cudaStream_t stream) {
  if ((size_t)red_grid() * kMaxTermsPerPass * 2 > scratch_doubles) return cudaErrorInvalidValue;
  std::vector<char> used(n_terms, 0);
  for (int t0 = 0; t0 < n_terms; t0++) {
    if (used[t0]) continue;
    TermPass tp{};
    TermOut to{};
    tp.x = terms[t0].x_mask;
    tp.h = tp.x ? 63 - __builtin_clzll(tp.x) : -1;
    for (int t = t0; t < n_terms && tp.nt < kMaxTermsPerPass; t++) {
      if (used[t] || terms[t].x_mask != tp.x) continue;
      used[t] = 1;
      tp.z[tp.nt] = terms[t].z_mask;
      to.dst[tp.nt] = t;
      to.ny[tp.nt] = __builtin_popcountll(terms[t].x_mask & terms[t].z_mask);
      tp.nt++;
    }
    to.nt = tp.nt;
    uint64_t count = tp.h >= 0 ? (1ull << (n - 1)) : (1ull << n);
    uint64_t g = (count + kRedThreads - 1) / kRedThreads;
    int grid = (int)(g < (uint64_t)red_grid() ? g : (uint64_t)red_grid());
    k_expect_terms<R><<<grid, kRedThreads, 0, stream>>>(state, n, tp, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finish_terms<<<1, 32, 0, stream>>>(scratch, grid, tp.h >= 0 ? 1 : 0, to, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t launch_expect_z_all<float>(const Cx<float>*, int, double*, size_t, double*, cudaStream_t);
template cudaError_t launch_expect_z_all<double>(const Cx<double>*, int, double*, size_t, double*, cudaStream_t);
template cudaError_t launch_expect_terms<float>(const Cx<float>*, int, const sv_pauli_term*, int, double*, size_t,
                                                double*, cudaStream_t);
template cudaError_t launch_expect_terms<double>(const Cx<double>*, int, const sv_pauli_term*, int, double*, size_t,
                                                 double*, cudaStream_t);

}  // namespace sv
