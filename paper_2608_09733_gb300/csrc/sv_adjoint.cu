// sv_adjoint.cu -- batched kernels of the adjoint (reverse-mode) gradient.
//
// Objective f(theta) = <0|U^dag(theta) H U(theta)|0> (Sec. 4.2).  With
// psi_k the state after gate k and lambda_k = U_{k+1}^dag ... U_N^dag H psi_N,
// a gate U_k = exp(-i theta G_k / 2) contributes
//     df/dtheta_k = 2 Re <lambda_k| dU_k/dtheta |psi_{k-1}> = Im <lambda_k|G_k|psi_k>,
// and the sweep walks back with psi <- U_k^dag psi, lambda <- U_k^dag lambda.
// (The paper differentiates through custom backward rules of each gate,
// Sec. 5.3; this is the tape-free form of the same reverse accumulation.)
//
// B states of one template run side by side (Sec. 4.1 BatchSV): grid.y is the
// state, grid.x the CTAs of one state.  A tile of psi and the same tile of
// lambda are gathered into shared memory; each op of a reverse program adds its
// gradient term over the tile and un-applies itself from both buffers in the
// same pass.  Per-CTA gradient partials go to a scratch array and are added in
// a fixed order by a second kernel.
#include <cuda_runtime.h>

#include "sv_internal.h"

namespace sv {
namespace {

template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ Cx<R> cfma(Cx<R> a, Cx<R> b, Cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
template <typename R>
__device__ __forceinline__ Cx<R> conjx(Cx<R> a) {
  return {a.re, -a.im};
}
// Im(conj(l) * g)
template <typename R>
__device__ __forceinline__ R im_cdot(Cx<R> l, Cx<R> g) {
  return l.re * g.im - l.im * g.re;
}

__device__ __forceinline__ uint32_t ins0(uint32_t x, int p) {
  uint32_t lo = x & ((1u << p) - 1u);
  return ((x >> p) << (p + 1)) | lo;
}
__device__ __forceinline__ uint64_t ins0_64(uint64_t x, int p) {
  uint64_t lo = x & ((1ull << p) - 1ull);
  return ((x >> p) << (p + 1)) | lo;
}

__device__ __forceinline__ uint64_t local_offset(uint32_t l, const BatchHeader& h) {
  uint64_t off = l & ((1u << h.L) - 1u);
#pragma unroll
  for (int i = 0; i < kMaxTileQ; i++) {
    if (i >= h.m) break;
    if (i >= h.L && ((l >> i) & 1u)) off |= 1ull << h.tq[i];
  }
  return off;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Element (r, c) of the op's matrix, or of its conjugate transpose.
template <typename R>
__device__ __forceinline__ Cx<R> mel(const Cx<R>* M, int d, int r, int c, bool dag) {
  return dag ? conjx(M[c * d + r]) : M[r * d + c];
}

// ---------------------------------------------------------------- dense d = 2, 4

template <typename R, int K, bool REV>
__device__ __forceinline__ void bop_dense(Cx<R>* sp, Cx<R>* sl, int tsz, const BOp& op, const Cx<R>* M,
                                          const Cx<R>* G, R& acc) {
  constexpr int D = 1 << K;
  const bool dag = op.dagger;
  for (uint32_t g = threadIdx.x; g < (uint32_t)(tsz >> K); g += blockDim.x) {
    uint32_t b = g;
#pragma unroll
    for (int i = 0; i < K; i++) b = ins0(b, op.spos[i]);
    if ((b & op.lmask) != op.lval) continue;
    uint32_t idx[D];
#pragma unroll
    for (int j = 0; j < D; j++) {
      uint32_t x = b;
#pragma unroll
      for (int i = 0; i < K; i++)
        if ((j >> i) & 1) x |= 1u << op.pos[i];
      idx[j] = x;
    }
    Cx<R> p[D];
#pragma unroll
    for (int j = 0; j < D; j++) p[j] = sp[idx[j]];
    if (REV) {
      Cx<R> l[D];
#pragma unroll
      for (int j = 0; j < D; j++) l[j] = sl[idx[j]];
      if (op.grad) {
#pragma unroll
        for (int r = 0; r < D; r++) {
          Cx<R> gp = {R(0), R(0)};
#pragma unroll
          for (int c = 0; c < D; c++) gp = cfma(G[r * D + c], p[c], gp);
          acc += im_cdot(l[r], gp);
        }
      }
#pragma unroll
      for (int r = 0; r < D; r++) {
        Cx<R> a = {R(0), R(0)};
#pragma unroll
        for (int c = 0; c < D; c++) a = cfma(mel(M, D, r, c, dag), l[c], a);
        sl[idx[r]] = a;
      }
    }
#pragma unroll
    for (int r = 0; r < D; r++) {
      Cx<R> a = {R(0), R(0)};
#pragma unroll
      for (int c = 0; c < D; c++) a = cfma(mel(M, D, r, c, dag), p[c], a);
      sp[idx[r]] = a;
    }
  }
}

template <typename R, bool REV>
__device__ __forceinline__ void bop_diag(Cx<R>* sp, Cx<R>* sl, int tsz, const BOp& op, const Cx<R>* M,
                                         const Cx<R>* G, uint64_t base, R& acc) {
  uint32_t xi = 0;
  for (int i = 0; i < op.k; i++)
    if (op.pos[i] == 0xFF) xi |= (uint32_t)((base >> op.gq[i]) & 1ull) << i;
  const bool dag = op.dagger;
  for (uint32_t a = threadIdx.x; a < (uint32_t)tsz; a += blockDim.x) {
    if ((a & op.lmask) != op.lval) continue;
    uint32_t di = xi;
    for (int i = 0; i < op.k; i++)
      if (op.pos[i] != 0xFF) di |= ((a >> op.pos[i]) & 1u) << i;
    Cx<R> u = dag ? conjx(M[di]) : M[di];
    Cx<R> p = sp[a];
    if (REV) {
      Cx<R> l = sl[a];
      if (op.grad) acc += im_cdot(l, cmul(G[di], p));
      sl[a] = cmul(u, l);
    }
    sp[a] = cmul(u, p);
  }
}

template <typename R, bool REV>
__device__ __forceinline__ void bop_antidiag(Cx<R>* sp, Cx<R>* sl, int tsz, const BOp& op, const Cx<R>* M) {
  const int p = op.pos[0];
  // [[0, a], [b, 0]]; its conjugate transpose is [[0, conj b], [conj a, 0]]
  Cx<R> a = op.dagger ? conjx(M[1]) : M[0];
  Cx<R> bb = op.dagger ? conjx(M[0]) : M[1];
  for (uint32_t g = threadIdx.x; g < (uint32_t)(tsz >> 1); g += blockDim.x) {
    uint32_t i0 = ins0(g, p);
    if ((i0 & op.lmask) != op.lval) continue;
    uint32_t i1 = i0 | (1u << p);
    Cx<R> v0 = sp[i0], v1 = sp[i1];
    sp[i0] = cmul(a, v1);
    sp[i1] = cmul(bb, v0);
    if (REV) {
      Cx<R> w0 = sl[i0], w1 = sl[i1];
      sl[i0] = cmul(a, w1);
      sl[i1] = cmul(bb, w0);
    }
  }
}

template <typename R, bool REV>
__device__ __forceinline__ void bop_swap(Cx<R>* sp, Cx<R>* sl, int tsz, const BOp& op) {
  for (uint32_t g = threadIdx.x; g < (uint32_t)(tsz >> 2); g += blockDim.x) {
    uint32_t b = ins0(ins0(g, op.spos[0]), op.spos[1]);
    if ((b & op.lmask) != op.lval) continue;
    uint32_t i01 = b | (1u << op.pos[0]), i10 = b | (1u << op.pos[1]);
    Cx<R> t = sp[i01];
    sp[i01] = sp[i10];
    sp[i10] = t;
    if (REV) {
      t = sl[i01];
      sl[i01] = sl[i10];
      sl[i10] = t;
    }
  }
}

template <typename R, bool REV>
__global__ void __launch_bounds__(256) k_batch_sweep(Cx<R>* __restrict__ psi, Cx<R>* __restrict__ lam,
                                                     const Cx<R>* __restrict__ table, double* __restrict__ gscratch,
                                                     const __grid_constant__ BatchProgram<R> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchHeader& h = P.h;
  const int tsz = 1 << h.m;
  Cx<R>* sp = reinterpret_cast<Cx<R>*>(smem_raw);
  Cx<R>* sl = sp + (REV ? tsz : 0);
  __shared__ double gacc[kBatchGacc][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kBatchGacc * 8; i += blockDim.x) gacc[i / 8][i % 8] = 0.0;
  const int bidx = blockIdx.y;
  Cx<R>* ps = psi + ((uint64_t)bidx << h.n);
  Cx<R>* ls = REV ? lam + ((uint64_t)bidx << h.n) : nullptr;
  constexpr int A = 16 / sizeof(Cx<R>);
  const int nvec = tsz / A;
  const uint64_t ntiles = 1ull << (h.n - h.m);
  __syncthreads();
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    uint64_t base = tile;
    for (int i = 0; i < h.m; i++) base = ins0_64(base, h.tq[i]);
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
      uint64_t off = local_offset((uint32_t)(v * A), h);
      reinterpret_cast<uint4*>(sp)[v] = *reinterpret_cast<const uint4*>(ps + (base + off));
      if (REV) reinterpret_cast<uint4*>(sl)[v] = *reinterpret_cast<const uint4*>(ls + (base + off));
    }
    __syncthreads();
    for (int o = 0; o < h.nops; o++) {
      const BOp& op = P.ops[o];
      if ((base & op.xmask) != op.xval) continue;  // uniform over the block
      const Cx<R>* M = op.table ? table + ((uint64_t)op.coef * h.batch + bidx) * kTableStride : P.pool + op.coef;
      const Cx<R>* G = P.pool + op.gen;
      R acc = R(0);
      switch (op.kind) {
        case OPK_DENSE:
          if (op.k == 1)
            bop_dense<R, 1, REV>(sp, sl, tsz, op, M, G, acc);
          else
            bop_dense<R, 2, REV>(sp, sl, tsz, op, M, G, acc);
          break;
        case OPK_DIAG: bop_diag<R, REV>(sp, sl, tsz, op, M, G, base, acc); break;
        case OPK_ANTIDIAG: bop_antidiag<R, REV>(sp, sl, tsz, op, M); break;
        case OPK_SWAP: bop_swap<R, REV>(sp, sl, tsz, op); break;
        default: break;
      }
      if (REV && op.grad) {
        double w = warp_sum((double)acc);
        if (lane == 0) gacc[op.gacc][warp] += w;
      }
      __syncthreads();
    }
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
      uint64_t off = local_offset((uint32_t)(v * A), h);
      *reinterpret_cast<uint4*>(ps + (base + off)) = reinterpret_cast<uint4*>(sp)[v];
      if (REV) *reinterpret_cast<uint4*>(ls + (base + off)) = reinterpret_cast<uint4*>(sl)[v];
    }
    __syncthreads();
  }
  if (REV) {
    for (int o = threadIdx.x; o < h.nops; o += blockDim.x) {
      const BOp& op = P.ops[o];
      if (!op.grad) continue;
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += gacc[op.gacc][w];
      gscratch[((uint64_t)bidx * h.ngrad_total + op.gidx) * gridDim.x + blockIdx.x] = s;
    }
  }
}

template <typename R>
__global__ void k_batch_init(Cx<R>* __restrict__ psi, uint64_t N, uint64_t total) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    Cx<R> v = {R((i & (N - 1)) == 0 ? 1 : 0), R(0)};
    psi[i] = v;
  }
}

constexpr int kMaxPauliGroup = 32;
struct PauliGroup {
  uint64_t x;
  int nt;
  uint64_t z[kMaxPauliGroup];
  double c[kMaxPauliGroup];
  int ny[kMaxPauliGroup];
};

// lam[i] (+)= sum_j c_j (P_j psi)[i],  (P psi)[i] = i^{nY} (-1)^{popc((i^x) & z)} psi[i ^ x]
template <typename R>
__global__ void __launch_bounds__(256) k_pauli_accum(const Cx<R>* __restrict__ psi, Cx<R>* __restrict__ lam, int n,
                                                     uint64_t total, PauliGroup pg, int accumulate) {
  const uint64_t mask = (1ull << n) - 1ull;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t li = i & mask;
    const uint64_t src = li ^ pg.x;
    Cx<R> v = psi[(i & ~mask) | src];
    double re = 0.0, im = 0.0;  // sum_j c_j i^{nY_j} (-1)^{popc(src & z_j)}
    for (int j = 0; j < pg.nt; j++) {
      double s = (__popcll(src & pg.z[j]) & 1) ? -pg.c[j] : pg.c[j];
      switch (pg.ny[j] & 3) {
        case 0: re += s; break;
        case 1: im += s; break;
        case 2: re -= s; break;
        default: im -= s; break;
      }
    }
    Cx<R> f = {(R)re, (R)im};
    Cx<R> add = cmul(f, v);
    if (accumulate) {
      Cx<R> o = lam[i];
      add.re += o.re;
      add.im += o.im;
    }
    lam[i] = add;
  }
}

constexpr int kDotThreads = 256;
constexpr int kDotGridX = 16;

template <typename R>
__global__ void __launch_bounds__(kDotThreads) k_batch_dot(const Cx<R>* __restrict__ psi, const Cx<R>* __restrict__ lam,
                                                           int n, double* __restrict__ partials) {
  __shared__ double red[kDotThreads / 32];
  const uint64_t N = 1ull << n;
  const Cx<R>* p = psi + ((uint64_t)blockIdx.y << n);
  const Cx<R>* l = lam + ((uint64_t)blockIdx.y << n);
  double acc = 0.0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N;) {
    R run = R(0);
    for (int r = 0; r < 64 && i < N; r++, i += (uint64_t)gridDim.x * blockDim.x) {
      Cx<R> a = p[i], b = l[i];
      run += a.re * b.re + a.im * b.im;  // Re(conj(a) b)
    }
    acc += (double)run;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kDotThreads / 32; w++) s += red[w];
    partials[(uint64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_sum_rows(const double* __restrict__ in, int rows, int cols, double* __restrict__ out) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < cols; c++) s += in[(uint64_t)r * cols + c];
    out[r] = s;
  }
}

}  // namespace

int batch_grid_x(int n, int m, int batch) {
  // about four resident CTAs per SM over the whole batch, at most one per tile
  int want = (device_sm_count() * 4 + batch - 1) / batch;
  uint64_t tiles = 1ull << (n - m);
  if ((uint64_t)want > tiles) want = (int)tiles;
  return want < 1 ? 1 : want;
}

template <typename R>
cudaError_t launch_batch_sweep(Cx<R>* psi, Cx<R>* lam, const Cx<R>* table, double* gscratch, int grid_x,
                               const BatchProgram<R>& prog, bool reverse, cudaStream_t stream) {
  const int smem = (int)sizeof(Cx<R>) << prog.h.m << (reverse ? 1 : 0);
  static int configured[2][64] = {{0}};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  dim3 grid((unsigned)grid_x, (unsigned)prog.h.batch);
  if (reverse) {
    if (smem > 48 * 1024 && smem > configured[1][dev]) {
      cudaError_t e = cudaFuncSetAttribute(k_batch_sweep<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      configured[1][dev] = smem;
    }
    k_batch_sweep<R, true><<<grid, 256, smem, stream>>>(psi, lam, table, gscratch, prog);
  } else {
    if (smem > 48 * 1024 && smem > configured[0][dev]) {
      cudaError_t e =
          cudaFuncSetAttribute(k_batch_sweep<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      configured[0][dev] = smem;
    }
    k_batch_sweep<R, false><<<grid, 256, smem, stream>>>(psi, lam, table, gscratch, prog);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_batch_init(Cx<R>* psi, int n, int batch, cudaStream_t stream) {
  uint64_t total = (uint64_t)batch << n;
  uint64_t grid = (total + 255) / 256, cap = (uint64_t)device_sm_count() * 8;
  k_batch_init<R><<<(unsigned)(grid < cap ? grid : cap), 256, 0, stream>>>(psi, 1ull << n, total);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pauli_accum(const Cx<R>* psi, Cx<R>* lam, int n, int batch, uint64_t x, const uint64_t* z,
                               const double* c, int nt, bool accumulate, cudaStream_t stream) {
  for (int t0 = 0; t0 < nt; t0 += kMaxPauliGroup) {
    PauliGroup pg{};
    pg.x = x;
    pg.nt = nt - t0 < kMaxPauliGroup ? nt - t0 : kMaxPauliGroup;
    for (int j = 0; j < pg.nt; j++) {
      pg.z[j] = z[t0 + j];
      pg.c[j] = c[t0 + j];
      pg.ny[j] = __builtin_popcountll(x & z[t0 + j]);
    }
    uint64_t total = (uint64_t)batch << n;
    uint64_t grid = (total + 255) / 256, cap = (uint64_t)device_sm_count() * 8;
    k_pauli_accum<R><<<(unsigned)(grid < cap ? grid : cap), 256, 0, stream>>>(psi, lam, n, total, pg,
                                                                          (accumulate || t0 > 0) ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

size_t batch_dot_scratch_doubles(int batch) { return (size_t)batch * kDotGridX; }

template <typename R>
cudaError_t launch_batch_dot(const Cx<R>* psi, const Cx<R>* lam, int n, int batch, double* scratch, double* out,
                             cudaStream_t stream) {
  dim3 grid(kDotGridX, (unsigned)batch);
  k_batch_dot<R><<<grid, kDotThreads, 0, stream>>>(psi, lam, n, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_rows<<<(batch + 127) / 128, 128, 0, stream>>>(scratch, batch, kDotGridX, out);
  return cudaGetLastError();
}

cudaError_t launch_grad_finish(const double* gscratch, int batch, int ngrad, int grid_x, double* out,
                               cudaStream_t stream) {
  int rows = batch * ngrad;
  if (rows == 0) return cudaSuccess;
  int blocks = (rows + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_sum_rows<<<blocks, 256, 0, stream>>>(gscratch, rows, grid_x, out);
  return cudaGetLastError();
}

#define SV_INST(R)                                                                                                \
  template cudaError_t launch_batch_sweep<R>(Cx<R>*, Cx<R>*, const Cx<R>*, double*, int, const BatchProgram<R>&, \
                                             bool, cudaStream_t);                                                 \
  template cudaError_t launch_batch_init<R>(Cx<R>*, int, int, cudaStream_t);                                      \
  template cudaError_t launch_pauli_accum<R>(const Cx<R>*, Cx<R>*, int, int, uint64_t, const uint64_t*,           \
                                             const double*, int, bool, cudaStream_t);                             \
  template cudaError_t launch_batch_dot<R>(const Cx<R>*, const Cx<R>*, int, int, double*, double*, cudaStream_t);
SV_INST(float)
SV_INST(double)
#undef SV_INST

}  // namespace sv
