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

#include <algorithm>
#include <cstring>
#include <vector>

#include "sv_adjoint.h"
#include "sv_batch_ops.cuh"

namespace sv {
namespace {


template <typename R, bool REV>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1)
    k_batch_sweep(Cx<R>* __restrict__ psi, Cx<R>* __restrict__ lam, const Cx<R>* __restrict__ table,
                  double* __restrict__ gscratch, const __grid_constant__ BatchProgram<R> P) {
  batch_sweep_body<R, REV>(psi, lam, table, gscratch, P, BatchInterp<R, REV>{P});
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

// lam (+)= H psi for the X-masks whose qubits all lie in one tile: the tile of
// psi is gathered into shared memory, and each amplitude sums, over the pass's
// terms, c_j i^{nY_j} (-1)^{popc(src & z_j)} psi[src] with src = b ^ x_j
// (Sec. 4.4: P|b> = i^{nY} (-1)^{popc(b & z)} |b ^ x>).  Terms are sorted by
// x, so each partner amplitude is read once per distinct x.
constexpr int kPauliTileTerms = 96;
struct PauliTilePass {
  int32_t n, m, L, nterms;
  int32_t accumulate, pad;
  int8_t tq[16];                      // tile qubits, ascending; tq[i] = i for i < L
  uint32_t xl[kPauliTileTerms];       // x in local tile bits
  uint64_t xg[kPauliTileTerms];       // x in global bits
  uint64_t z[kPauliTileTerms];
  uint32_t zl[kPauliTileTerms];       // z in local tile bits
  uint8_t gend[kPauliTileTerms];      // at the first term of a run of equal xl: one past the run
  double cr[kPauliTileTerms], ci[kPauliTileTerms];  // c_j i^{nY_j}
  uint16_t orig[kPauliTileTerms];     // the term's index in the caller's list (per-state coefficients)
  uint8_t ny[kPauliTileTerms];        // nY_j mod 4
  int32_t nterms_all;                 // terms per state in the per-state coefficient rows
};

// The pass's coefficients in the state's precision (FP64 is a slow pipe on
// GB300), staged in shared memory by the kernel.
template <typename R>
struct PauliTileCoef {
  R cr, ci;
};

// With `rowc` (device, batch x nterms_all doubles) state b takes its own
// coefficients c_{b,j} in place of P.cr / P.ci.
template <typename R>
__global__ void __launch_bounds__(256) k_pauli_tiles(const Cx<R>* __restrict__ psi, Cx<R>* __restrict__ lam,
                                                     const __grid_constant__ PauliTilePass P, uint64_t ntiles,
                                                     const double* __restrict__ rowc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<R>* s = reinterpret_cast<Cx<R>*>(smem_raw);
  const int tsz = 1 << P.m;
  uint64_t* hi_off = reinterpret_cast<uint64_t*>(s + tsz);
  const int nhi = 1 << (P.m - P.L);
  __shared__ PauliTileCoef<R> cf[kPauliTileTerms];
  // the terms' masks, staged once (broadcast reads in the inner loop)
  // The sign (-1)^{popc((g ^ x) & z)} of a term splits into the tile-local
  // part popc(l & zl) and a part that is fixed over the tile (the bits
  // outside it, and x inside it): sc0[j], restaged per tile.
  __shared__ uint32_t sxl[kPauliTileTerms], szl[kPauliTileTerms];
  __shared__ uint8_t sgend[kPauliTileTerms], sc0[kPauliTileTerms];
  for (int j = threadIdx.x; j < P.nterms; j += blockDim.x) {
    sxl[j] = P.xl[j];
    szl[j] = P.zl[j];
    sgend[j] = P.gend[j];
  }
  uint64_t tile_mask = 0;
  for (int i = 0; i < P.m; i++) tile_mask |= 1ull << P.tq[i];
  for (int c = threadIdx.x; c < nhi; c += blockDim.x) {
    uint64_t off = 0;
    for (int i = P.L; i < P.m; i++)
      if (((uint32_t)c >> (i - P.L)) & 1u) off |= 1ull << P.tq[i];
    hi_off[c] = off;
  }
  if (!rowc)
    for (int j = threadIdx.x; j < P.nterms; j += blockDim.x) cf[j] = {(R)P.cr[j], (R)P.ci[j]};
  __syncthreads();
  uint64_t staged = ~0ull;  // state whose coefficients cf holds (per-state mode)
  const uint32_t lowmask = (1u << P.L) - 1u;
  const int per_state_log = P.n - P.m;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t b = tile >> per_state_log;
    uint64_t base = tile & ((1ull << per_state_log) - 1ull);
    for (int i = 0; i < P.m; i++) base = ins0_64(base, P.tq[i]);
    const uint64_t sbase = b << P.n;
    if (rowc && b != staged) {  // every thread sees the same b: uniform branch
      for (int j = threadIdx.x; j < P.nterms; j += blockDim.x) {
        const R c = (R)rowc[b * (uint64_t)P.nterms_all + P.orig[j]];
        const int ny = P.ny[j];
        cf[j] = {ny == 0 ? c : ny == 2 ? -c : R(0), ny == 1 ? c : ny == 3 ? -c : R(0)};
      }
      staged = b;
    }
    for (int l = threadIdx.x; l < tsz; l += blockDim.x)
      s[l] = psi[sbase + (base | hi_off[l >> P.L] | (l & lowmask))];
    for (int j = threadIdx.x; j < P.nterms; j += blockDim.x)
      sc0[j] = (uint8_t)((__popcll((base ^ P.xg[j]) & P.z[j] & ~tile_mask) + __popc(P.xl[j] & P.zl[j])) & 1);
    __syncthreads();
    // four amplitudes per thread: each term's masks and coefficient are read
    // once for all four, and the four sums are independent
    constexpr int A = 4;
    const int stride = (int)blockDim.x;
    for (int l0 = threadIdx.x; l0 < tsz; l0 += A * stride) {
      uint64_t g[A];
      R ar[A], ai[A];
#pragma unroll
      for (int k = 0; k < A; k++) {
        const int l = l0 + k * stride < tsz ? l0 + k * stride : l0;  // past the tile: a repeat, not stored
        g[k] = base | hi_off[l >> P.L] | (l & lowmask);
        ar[k] = ai[k] = R(0);
      }
      int lk[A];
#pragma unroll
      for (int k = 0; k < A; k++) lk[k] = l0 + k * stride < tsz ? l0 + k * stride : l0;
      for (int j = 0; j < P.nterms;) {
        const uint32_t xl = sxl[j];
        const int je = sgend[j];
        R fr[A], fi[A];
#pragma unroll
        for (int k = 0; k < A; k++) fr[k] = fi[k] = R(0);
        for (; j < je; j++) {
          const uint32_t zl = szl[j], c0 = sc0[j];
          const PauliTileCoef<R> c = cf[j];
#pragma unroll
          for (int k = 0; k < A; k++) {
            const bool neg = (__popc((uint32_t)lk[k] & zl) ^ c0) & 1u;
            fr[k] += neg ? -c.cr : c.cr;
            fi[k] += neg ? -c.ci : c.ci;
          }
        }
#pragma unroll
        for (int k = 0; k < A; k++) {
          const Cx<R> v = s[lk[k] ^ xl];
          ar[k] = fma(fr[k], v.re, fma(-fi[k], v.im, ar[k]));
          ai[k] = fma(fr[k], v.im, fma(fi[k], v.re, ai[k]));
        }
      }
#pragma unroll
      for (int k = 0; k < A; k++) {
        if (l0 + k * stride >= tsz) continue;
        Cx<R>* o = lam + sbase + g[k];
        if (P.accumulate) {
          const Cx<R> w = *o;
          ar[k] += w.re;
          ai[k] += w.im;
        }
        *o = Cx<R>{ar[k], ai[k]};
      }
    }
    __syncthreads();
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
                               const BatchProgram<R>& prog, bool reverse, cudaStream_t stream, const JitKernel* jit) {
  const int smem = ((int)sizeof(Cx<R>) << prog.h.m << (reverse ? 1 : 0)) + (8 << (prog.h.m - prog.h.L)) +
                   (int)sizeof(Cx<R>) * prog.h.scoef;
  // one thread per register group of the tile (16 amplitudes), 32..256
  const int g = prog.h.m - kRegQ;
  const int threads = g >= 5 && g < 8 ? (1 << g) : 256;
  if (jit)
    return jit_batch_launch(jit, psi, lam, table, gscratch, &prog, (unsigned)grid_x, (unsigned)prog.h.batch,
                            (unsigned)threads, (size_t)smem, stream);
  static int configured[2][64] = {{0}};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  dim3 grid((unsigned)grid_x, (unsigned)prog.h.batch);
  auto go = [&](auto kernel, int which) -> cudaError_t {
    if (smem > 48 * 1024 && smem > configured[which][dev]) {
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      configured[which][dev] = smem;
    }
    kernel<<<grid, threads, smem, stream>>>(psi, lam, table, gscratch, prog);
    return cudaGetLastError();
  };
  return reverse ? go(k_batch_sweep<R, true>, 0) : go(k_batch_sweep<R, false>, 1);
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

// lam (+)= sum_j c_j P_j psi: the X-masks are covered greedily by tiles of m
// qubits that always hold the lowest L (coalesced runs); all terms whose x
// lies in a tile are applied in that tile's pass.  Masks no tile can hold
// fall back to one pass per mask (launch_pauli_accum).
template <typename R>
cudaError_t launch_pauli_tiles(const Cx<R>* psi, Cx<R>* lam, int n, int batch, const sv_pauli_term* terms,
                               int nterms, bool accumulate, const double* rowc, cudaStream_t stream) {
  const int L = std::min(n, sizeof(R) == 4 ? 5 : 4);
  const int m = std::min(n, sizeof(R) == 4 ? 13 : 12);  // 64 KiB tiles
  std::vector<int> idx(nterms);
  for (int t = 0; t < nterms; t++) idx[t] = t;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return terms[a].x_mask < terms[b].x_mask; });
  const uint64_t low = (1ull << L) - 1ull;
  std::vector<char> done(nterms, 0);
  bool acc = accumulate;
  int remaining = nterms;
  while (remaining > 0) {
    // tile qubits: the low L, then the qubits of uncovered masks that fit
    uint64_t T = low;
    for (int t : idx) {
      if (done[t]) continue;
      const uint64_t u = T | terms[t].x_mask;
      if (__builtin_popcountll(u) <= m) T = u;
    }
    bool any = false;
    for (int t : idx)
      if (!done[t] && (terms[t].x_mask & ~T) == 0) any = true;
    if (!any) break;  // the rest need wider tiles
    for (int q = 0; q < n && __builtin_popcountll(T) < m; q++) T |= 1ull << q;
    PauliTilePass P;
    std::memset(&P, 0, sizeof(P));
    P.n = n;
    P.m = m;
    P.L = L;
    P.nterms_all = nterms;
    int loc[64], k = 0;
    for (int q = 0; q < n; q++)
      if ((T >> q) & 1ull) {
        loc[q] = k;
        P.tq[k++] = (int8_t)q;
      }
    auto flush = [&]() -> cudaError_t {
      if (!P.nterms) return cudaSuccess;
      for (int j = P.nterms - 1; j >= 0; j--)  // runs of equal xl
        P.gend[j] = (uint8_t)(j + 1 < P.nterms && P.xl[j + 1] == P.xl[j] ? P.gend[j + 1] : j + 1);
      P.accumulate = acc ? 1 : 0;
      const uint64_t ntiles = (uint64_t)batch << (n - m);
      const int smem = (int)(sizeof(Cx<R>) << m) + (8 << (m - L));
      static int configured[64] = {0};
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
      if (smem > 48 * 1024 && smem > configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_pauli_tiles<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured[dev] = smem;
      }
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pauli_tiles<R>, 256, smem);
      uint64_t grid = (uint64_t)device_sm_count() * (per_sm > 0 ? per_sm : 1);
      if (grid > ntiles) grid = ntiles;
      k_pauli_tiles<R><<<(unsigned)grid, 256, smem, stream>>>(psi, lam, P, ntiles, rowc);
      acc = true;
      P.nterms = 0;
      return cudaGetLastError();
    };
    for (int t : idx) {
      if (done[t] || (terms[t].x_mask & ~T)) continue;
      if (P.nterms == kPauliTileTerms) {
        cudaError_t e = flush();
        if (e != cudaSuccess) return e;
      }
      const uint64_t x = terms[t].x_mask;
      uint32_t xl = 0;
      for (int q = 0; q < n; q++)
        if ((x >> q) & 1ull) xl |= 1u << loc[q];
      const int ny = __builtin_popcountll(x & terms[t].z_mask) & 3;  // i^{nY}
      const double c = terms[t].coeff;
      const int j = P.nterms++;
      P.xl[j] = xl;
      P.xg[j] = x;
      P.z[j] = terms[t].z_mask;
      uint32_t zl = 0;
      for (int q = 0; q < n; q++)
        if (((terms[t].z_mask >> q) & 1ull) && ((T >> q) & 1ull)) zl |= 1u << loc[q];
      P.zl[j] = zl;
      P.cr[j] = ny == 0 ? c : ny == 2 ? -c : 0.0;
      P.ci[j] = ny == 1 ? c : ny == 3 ? -c : 0.0;
      P.orig[j] = (uint16_t)t;
      P.ny[j] = (uint8_t)ny;
      done[t] = 1;
      remaining--;
    }
    cudaError_t e = flush();
    if (e != cudaSuccess) return e;
  }
  // masks wider than a tile: one pass per mask (shared coefficients only)
  if (rowc)
    for (int t = 0; t < nterms; t++)
      if (!done[t]) return cudaErrorNotSupported;
  for (int a = 0; a < nterms; a++) {
    const int t0 = idx[a];
    if (done[t0]) continue;
    std::vector<uint64_t> zs;
    std::vector<double> cs;
    for (int b2 = a; b2 < nterms; b2++) {
      const int t = idx[b2];
      if (!done[t] && terms[t].x_mask == terms[t0].x_mask) {
        done[t] = 1;
        zs.push_back(terms[t].z_mask);
        cs.push_back(terms[t].coeff);
      }
    }
    cudaError_t e = launch_pauli_accum<R>(psi, lam, n, batch, terms[t0].x_mask, zs.data(), cs.data(), (int)zs.size(),
                                          acc, stream);
    if (e != cudaSuccess) return e;
    acc = true;
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

// ---------------------------------------------------------------- device-side tables

namespace {

// One thread per (parameterised gate, state): the gate's matrix at the
// state's parameter value, in double precision (sincos), narrowed once, in
// the layout the host builds (d diagonal entries, or d x d row-major).
template <typename R>
__global__ void k_build_tables(const double* __restrict__ params, int npar, int batch,
                               const TableGate* __restrict__ gates, int ngates, Cx<R>* __restrict__ table) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)ngates * batch) return;
  const int pidx = (int)(i / batch), b = (int)(i % batch);
  const TableGate tg = gates[pidx];
  const double th = params[(size_t)b * npar + tg.slot];
  double s, c;
  sincos(0.5 * th, &s, &c);
  Cx<R>* row = table + (size_t)i * kTableStride;
  auto put = [&](int e, double re, double im) { row[e] = Cx<R>{(R)re, (R)im}; };
  switch (tg.type) {
    case SV_GATE_RX: put(0, c, 0); put(1, 0, -s); put(2, 0, -s); put(3, c, 0); break;
    case SV_GATE_RY: put(0, c, 0); put(1, -s, 0); put(2, s, 0); put(3, c, 0); break;
    case SV_GATE_RZ: put(0, c, -s); put(1, c, s); break;  // diagonal
    case SV_GATE_P: {                                      // diagonal
      double s1, c1;
      sincos(th, &s1, &c1);
      put(0, 1, 0);
      put(1, c1, s1);
      break;
    }
    case SV_GATE_RZZ: put(0, c, -s); put(1, c, s); put(2, c, s); put(3, c, -s); break;  // diagonal
    case SV_GATE_RXX:
    case SV_GATE_RYY: {  // cos I - i sin P(x)P; YY has -1 on its outer anti-diagonal corners
      const double outer = tg.type == SV_GATE_RXX ? 1.0 : -1.0;
      for (int e = 0; e < 16; e++) put(e, (e % 5 == 0) ? c : 0.0, 0.0);
      put(0 * 4 + 3, 0, -s * outer);
      put(3 * 4 + 0, 0, -s * outer);
      put(1 * 4 + 2, 0, -s);
      put(2 * 4 + 1, 0, -s);
      break;
    }
    case SV_GATE_EXC1: {  // identity except [[c, -s], [s, c]] on indices (1, 2)
      for (int e = 0; e < 16; e++) put(e, (e % 5 == 0) ? 1.0 : 0.0, 0.0);
      put(1 * 4 + 1, c, 0);
      put(1 * 4 + 2, -s, 0);
      put(2 * 4 + 1, s, 0);
      put(2 * 4 + 2, c, 0);
      break;
    }
    default: break;
  }
}

// out[b, p] = sum of g[b, pidx] over the parameterised gates pidx bound to
// slot p (in gate order, so the sums do not depend on scheduling).
__global__ void k_scatter_grad(const double* __restrict__ g, int batch, int ngrad, const int* __restrict__ slot,
                               int npar, double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double* o = out + (size_t)b * npar;
  for (int p = 0; p < npar; p++) o[p] = 0.0;
  for (int k = 0; k < ngrad; k++) o[slot[k]] += g[(size_t)b * ngrad + k];
}

}  // namespace

template <typename R>
cudaError_t launch_build_tables(const double* params, int npar, int batch, const TableGate* gates, int ngates,
                                Cx<R>* table, cudaStream_t stream) {
  const long long n = (long long)ngates * batch;
  if (n == 0) return cudaSuccess;
  k_build_tables<R><<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(params, npar, batch, gates, ngates, table);
  return cudaGetLastError();
}

cudaError_t launch_scatter_grad(const double* g, int batch, int ngrad, const int* slot, int npar, double* out,
                                cudaStream_t stream) {
  if (batch == 0 || npar == 0) return cudaSuccess;
  k_scatter_grad<<<(batch + 127) / 128, 128, 0, stream>>>(g, batch, ngrad, slot, npar, out);
  return cudaGetLastError();
}

#define SV_INST(R)                                                                                                \
  template cudaError_t launch_build_tables<R>(const double*, int, int, const TableGate*, int, Cx<R>*,              \
                                              cudaStream_t);                                                      \
  template cudaError_t launch_batch_sweep<R>(Cx<R>*, Cx<R>*, const Cx<R>*, double*, int, const BatchProgram<R>&, \
                                             bool, cudaStream_t, const JitKernel*);                               \
  template cudaError_t launch_batch_init<R>(Cx<R>*, int, int, cudaStream_t);                                      \
  template cudaError_t launch_pauli_accum<R>(const Cx<R>*, Cx<R>*, int, int, uint64_t, const uint64_t*,           \
                                             const double*, int, bool, cudaStream_t);                             \
  template cudaError_t launch_pauli_tiles<R>(const Cx<R>*, Cx<R>*, int, int, const sv_pauli_term*, int, bool,      \
                                             const double*, cudaStream_t);                                        \
  template cudaError_t launch_batch_dot<R>(const Cx<R>*, const Cx<R>*, int, int, double*, double*, cudaStream_t);
SV_INST(float)
SV_INST(double)
#undef SV_INST

}  // namespace sv
