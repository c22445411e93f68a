// sv_sweep.cu -- gate application kernels for sm_103a.
//
// One launch makes one pass over the state (the "sweep").  The state is cut
// into tiles of 2^m amplitudes; a tile is the set of amplitudes whose bits
// outside the tile qubits tq[] are fixed, i.e. the paper's group of amplitudes
// "that differ only on the target qubits" (Sec. 5.3), widened from the k
// targets of one gate to the m qubits of every operation the pass applies.
// Group members are found by bit insertion instead of the paper's index table
// I_T (no 2^n integer array is stored).  The low L tile qubits are 0..L-1, so a
// tile is 2^(m-L) contiguous runs of 2^L amplitudes (256 bytes): each run is
// read and written with coalesced 16-byte accesses.
//
// Inside the tile every operation of the program is applied in shared memory:
// dense k <= 5 matrices (single gates or the paper's fused blocks), real
// matrices with half the multiplies (Sec. 5.3: a real gate needs 2 real
// products, a complex one 4), diagonal gates (no amplitude moves), and the
// permutation gates X/CNOT/SWAP (Sec. 9.2: diagonal and permutation paths).
#include <cuda_runtime.h>

#include "sv_internal.h"

namespace sv {

namespace {

template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ Cx<R> cfma(Cx<R> a, Cx<R> b, Cx<R> acc) {  // acc + a*b
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}

__device__ __forceinline__ uint32_t ins0(uint32_t x, int p) {  // insert a zero bit at p
  uint32_t lo = x & ((1u << p) - 1u);
  return ((x >> p) << (p + 1)) | lo;
}
__device__ __forceinline__ uint64_t ins0_64(uint64_t x, int p) {
  uint64_t lo = x & ((1ull << p) - 1ull);
  return ((x >> p) << (p + 1)) | lo;
}

// Offset of local amplitude l (m bits) from the tile base in the global state.
__device__ __forceinline__ uint64_t local_offset(uint32_t l, const ProgramHeader& h) {
  uint64_t off = l & ((1u << h.L) - 1u);
#pragma unroll
  for (int i = 0; i < kMaxTileQ; i++) {
    if (i >= h.m) break;
    if (i >= h.L && ((l >> i) & 1u)) off |= 1ull << h.tq[i];
  }
  return off;
}

// ---------------------------------------------------------------- ops

template <typename R>
__device__ __forceinline__ void op_dense1(Cx<R>* s, int tsz, const DevOp& op, const Cx<R>* cf, bool real) {
  const int p = op.pos[0];
  const Cx<R> u00 = cf[0], u01 = cf[1], u10 = cf[2], u11 = cf[3];
  for (uint32_t g = threadIdx.x; g < (uint32_t)(tsz >> 1); g += blockDim.x) {
    uint32_t i0 = ins0(g, p);
    if ((i0 & op.lmask) != op.lval) continue;
    uint32_t i1 = i0 | (1u << p);
    Cx<R> a = s[i0], b = s[i1];
    Cx<R> o0, o1;
    if (real) {
      o0 = {fma(u00.re, a.re, u01.re * b.re), fma(u00.re, a.im, u01.re * b.im)};
      o1 = {fma(u10.re, a.re, u11.re * b.re), fma(u10.re, a.im, u11.re * b.im)};
    } else {
      o0 = cfma(u01, b, cmul(u00, a));
      o1 = cfma(u11, b, cmul(u10, a));
    }
    s[i0] = o0;
    s[i1] = o1;
  }
}

template <typename R>
__device__ __forceinline__ void op_antidiag(Cx<R>* s, int tsz, const DevOp& op, const Cx<R>* cf) {
  const int p = op.pos[0];
  const Cx<R> a01 = cf[0], a10 = cf[1];
  for (uint32_t g = threadIdx.x; g < (uint32_t)(tsz >> 1); g += blockDim.x) {
    uint32_t i0 = ins0(g, p);
    if ((i0 & op.lmask) != op.lval) continue;
    uint32_t i1 = i0 | (1u << p);
    Cx<R> a = s[i0], b = s[i1];
    s[i0] = cmul(a01, b);
    s[i1] = cmul(a10, a);
  }
}

template <typename R>
__device__ __forceinline__ void op_swap(Cx<R>* s, int tsz, const DevOp& op) {
  const int p0 = op.pos[0], p1 = op.pos[1];
  const int q0 = op.spos[0], q1 = op.spos[1];
  for (uint32_t g = threadIdx.x; g < (uint32_t)(tsz >> 2); g += blockDim.x) {
    uint32_t b = ins0(ins0(g, q0), q1);
    if ((b & op.lmask) != op.lval) continue;
    uint32_t i01 = b | (1u << p0), i10 = b | (1u << p1);
    Cx<R> t = s[i01];
    s[i01] = s[i10];
    s[i10] = t;
  }
}

template <typename R, int K>
__device__ __forceinline__ void op_denseK(Cx<R>* s, int tsz, const DevOp& op, const Cx<R>* cf, bool real) {
  constexpr int D = 1 << K;
  uint32_t bit[K];
#pragma unroll
  for (int i = 0; i < K; i++) bit[i] = 1u << op.pos[i];
  for (uint32_t g = threadIdx.x; g < (uint32_t)(tsz >> K); g += blockDim.x) {
    uint32_t b = g;
#pragma unroll
    for (int i = 0; i < K; i++) b = ins0(b, op.spos[i]);
    if ((b & op.lmask) != op.lval) continue;
    Cx<R> v[D];
#pragma unroll
    for (int j = 0; j < D; j++) {
      uint32_t x = b;
#pragma unroll
      for (int i = 0; i < K; i++)
        if ((j >> i) & 1) x |= bit[i];
      v[j] = s[x];
    }
#pragma unroll 1
    for (int r = 0; r < D; r++) {
      Cx<R> acc = {R(0), R(0)};
      const Cx<R>* row = cf + r * D;
      if (real) {
#pragma unroll
        for (int c = 0; c < D; c++) {
          acc.re = fma(row[c].re, v[c].re, acc.re);
          acc.im = fma(row[c].re, v[c].im, acc.im);
        }
      } else {
#pragma unroll
        for (int c = 0; c < D; c++) acc = cfma(row[c], v[c], acc);
      }
      uint32_t x = b;
#pragma unroll
      for (int i = 0; i < K; i++)
        if ((r >> i) & 1) x |= bit[i];
      s[x] = acc;
    }
  }
}

template <typename R>
__device__ __forceinline__ void op_diag(Cx<R>* s, int tsz, const DevOp& op, const Cx<R>* cf, uint64_t base) {
  // external matrix bits are fixed for the whole tile
  uint32_t xi = 0;
  for (int i = 0; i < op.k; i++)
    if (op.pos[i] == 0xFF) xi |= (uint32_t)((base >> op.gq[i]) & 1ull) << i;
  for (uint32_t a = threadIdx.x; a < (uint32_t)tsz; a += blockDim.x) {
    if ((a & op.lmask) != op.lval) continue;
    uint32_t di = xi;
    for (int i = 0; i < op.k; i++)
      if (op.pos[i] != 0xFF) di |= ((a >> op.pos[i]) & 1u) << i;
    s[a] = cmul(cf[di], s[a]);
  }
}

// ---------------------------------------------------------------- kernels

// KMAX: widest dense operation the program holds (the host picks the variant,
// so programs of one- and two-qubit gates do not pay the registers of k = 5).
template <typename R, int KMAX>
__global__ void __launch_bounds__(256) k_sweep(Cx<R>* __restrict__ state, const __grid_constant__ SweepProgram<R> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<R>* s = reinterpret_cast<Cx<R>*>(smem_raw);
  const ProgramHeader& h = P.h;
  const int tsz = 1 << h.m;
  constexpr int A = 16 / sizeof(Cx<R>);  // amplitudes per 16-byte access
  const int nvec = tsz / A;
  const uint64_t ntiles = 1ull << (h.n - h.m);
  uint4* s4 = reinterpret_cast<uint4*>(s);
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    uint64_t base = tile;
    for (int i = 0; i < h.m; i++) base = ins0_64(base, h.tq[i]);
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
      uint64_t off = local_offset((uint32_t)(v * A), h);
      s4[v] = *reinterpret_cast<const uint4*>(state + (base + off));
    }
    __syncthreads();
    for (int o = 0; o < h.nops; o++) {
      const DevOp& op = P.ops[o];
      if ((base & op.xmask) != op.xval) continue;  // same for the whole block
      const Cx<R>* cf = P.coef + op.coef;
      switch (op.kind) {
        case OPK_DENSE:
        case OPK_REAL: {
          bool real = op.kind == OPK_REAL;
          switch (op.k) {
            case 1: op_dense1<R>(s, tsz, op, cf, real); break;
            case 2: op_denseK<R, 2>(s, tsz, op, cf, real); break;
            case 3: if constexpr (KMAX >= 3) op_denseK<R, 3>(s, tsz, op, cf, false); break;
            case 4: if constexpr (KMAX >= 4) op_denseK<R, 4>(s, tsz, op, cf, false); break;
            default: if constexpr (KMAX >= 5) op_denseK<R, 5>(s, tsz, op, cf, false); break;
          }
          break;
        }
        case OPK_DIAG: op_diag<R>(s, tsz, op, cf, base); break;
        case OPK_ANTIDIAG: op_antidiag<R>(s, tsz, op, cf); break;
        case OPK_SWAP: op_swap<R>(s, tsz, op); break;
        default: break;
      }
      __syncthreads();
    }
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
      uint64_t off = local_offset((uint32_t)(v * A), h);
      *reinterpret_cast<uint4*>(state + (base + off)) = s4[v];
    }
    __syncthreads();
  }
}

template <typename R>
__global__ void k_init_basis(Cx<R>* __restrict__ state, uint64_t N, uint64_t index) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    Cx<R> v = {R(i == index ? 1 : 0), R(0)};
    state[i] = v;
  }
}

}  // namespace

int device_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <typename R, int KMAX>
static cudaError_t launch_sweep_k(Cx<R>* state, const SweepProgram<R>& prog, cudaStream_t stream) {
  const int smem = (int)sizeof(Cx<R>) << prog.h.m;
  // raise the dynamic shared-memory limit to what this launch needs (per device)
  static int configured_bytes[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem > 48 * 1024 && smem > configured_bytes[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep<R, KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured_bytes[dev] = smem;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<R, KMAX>, 256, smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t ntiles = 1ull << (prog.h.n - prog.h.m);
  uint64_t grid = (uint64_t)device_sm_count() * per_sm;
  if (grid > ntiles) grid = ntiles;
  k_sweep<R, KMAX><<<(unsigned)grid, 256, smem, stream>>>(state, prog);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sweep(Cx<R>* state, const SweepProgram<R>& prog, cudaStream_t stream) {
  int kmax = 1;
  for (int o = 0; o < prog.h.nops; o++) {
    const DevOp& op = prog.ops[o];
    if ((op.kind == OPK_DENSE || op.kind == OPK_REAL) && op.k > kmax) kmax = op.k;
  }
  if (kmax <= 2) return launch_sweep_k<R, 2>(state, prog, stream);
  if (kmax == 3) return launch_sweep_k<R, 3>(state, prog, stream);
  return launch_sweep_k<R, 5>(state, prog, stream);
}

template <typename R>
cudaError_t launch_init_basis(Cx<R>* state, int n, uint64_t index, cudaStream_t stream) {
  const uint64_t N = 1ull << n;
  uint64_t grid = (N + 255) / 256;
  uint64_t cap = (uint64_t)device_sm_count() * 8;
  if (grid > cap) grid = cap;
  k_init_basis<R><<<(unsigned)grid, 256, 0, stream>>>(state, N, index);
  return cudaGetLastError();
}

template cudaError_t launch_sweep<float>(Cx<float>*, const SweepProgram<float>&, cudaStream_t);
template cudaError_t launch_sweep<double>(Cx<double>*, const SweepProgram<double>&, cudaStream_t);
template cudaError_t launch_init_basis<float>(Cx<float>*, int, uint64_t, cudaStream_t);
template cudaError_t launch_init_basis<double>(Cx<double>*, int, uint64_t, cudaStream_t);

}  // namespace sv
