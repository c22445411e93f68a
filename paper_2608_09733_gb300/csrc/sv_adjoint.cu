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

// Shared-memory slot of local amplitude l (XOR swizzle of 16-byte granules,
// the same as the single-state sweep).
template <typename R>
__device__ __forceinline__ uint32_t sw(uint32_t l) {
  if constexpr (sizeof(Cx<R>) == 8)
    return l ^ ((l >> 3) & 14u);
  else
    return l ^ ((l >> 3) & 7u);
}

// Asynchronous 16-byte global -> shared copy; cp_async_commit_wait_all()
// waits for all of this thread's copies.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
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
      idx[j] = sw<R>(x);
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
    const uint32_t pa = sw<R>(a);
    Cx<R> p = sp[pa];
    if (REV) {
      Cx<R> l = sl[pa];
      if (op.grad) acc += im_cdot(l, cmul(G[di], p));
      sl[pa] = cmul(u, l);
    }
    sp[pa] = cmul(u, p);
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
    uint32_t i1 = sw<R>(i0 | (1u << p));
    i0 = sw<R>(i0);
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
    uint32_t i01 = sw<R>(b | (1u << op.pos[0])), i10 = sw<R>(b | (1u << op.pos[1]));
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

// ---------------------------------------------------------------- register phases
//
// As in the single-state sweep, a register phase gives each thread the 16
// amplitudes of four register qubits -- here of psi and, in reverse mode, of
// lambda -- and applies its ops with FMAs on registers.

constexpr int NR = 1 << kRegQ;

// Matrix element (r, c) of U (or U^dag) of dimension D.
template <typename R, int D>
__device__ __forceinline__ Cx<R> uel(const Cx<R>* M, int r, int c, bool dag) {
  return dag ? conjx(M[c * D + r]) : M[r * D + c];
}

template <typename R, int S, bool REV>
__device__ __forceinline__ void b_dense1(Cx<R> (&p)[NR], Cx<R> (&l)[NR], const BOp& op, const Cx<R>* M,
                                         const Cx<R>* G, R& acc) {
  const bool dag = op.dagger;
  const Cx<R> u00 = uel<R, 2>(M, 0, 0, dag), u01 = uel<R, 2>(M, 0, 1, dag);
  const Cx<R> u10 = uel<R, 2>(M, 1, 0, dag), u11 = uel<R, 2>(M, 1, 1, dag);
  const bool grad = REV && op.grad;
  const uint32_t rm = op.rmask, rv = op.rval;
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if (j & (1 << S)) continue;
    if ((j & rm) != rv) continue;
    const int j1 = j | (1 << S);
    const Cx<R> a = p[j], b = p[j1];
    if (grad) {
      const Cx<R> g0 = cfma(G[1], b, cmul(G[0], a)), g1 = cfma(G[3], b, cmul(G[2], a));
      acc += im_cdot(l[j], g0) + im_cdot(l[j1], g1);
    }
    p[j] = cfma(u01, b, cmul(u00, a));
    p[j1] = cfma(u11, b, cmul(u10, a));
    if (REV) {
      const Cx<R> c = l[j], d = l[j1];
      l[j] = cfma(u01, d, cmul(u00, c));
      l[j1] = cfma(u11, d, cmul(u10, c));
    }
  }
}

// A = register slot of matrix bit 0, B = of matrix bit 1.
template <typename R, int A, int B, bool REV>
__device__ __forceinline__ void b_dense2(Cx<R> (&p)[NR], Cx<R> (&l)[NR], const BOp& op, const Cx<R>* M,
                                         const Cx<R>* G, R& acc) {
  const bool dag = op.dagger;
  const bool grad = REV && op.grad;
  const uint32_t rm = op.rmask, rv = op.rval;
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if (j & ((1 << A) | (1 << B))) continue;
    if ((j & rm) != rv) continue;
    const int idx[4] = {j, j | (1 << A), j | (1 << B), j | (1 << A) | (1 << B)};
    Cx<R> x[4];
#pragma unroll
    for (int c = 0; c < 4; c++) x[c] = p[idx[c]];
    if (grad) {
#pragma unroll
      for (int r = 0; r < 4; r++) {
        Cx<R> g = cmul(G[r * 4], x[0]);
#pragma unroll
        for (int c = 1; c < 4; c++) g = cfma(G[r * 4 + c], x[c], g);
        acc += im_cdot(l[idx[r]], g);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
      Cx<R> o = cmul(uel<R, 4>(M, r, 0, dag), x[0]);
#pragma unroll
      for (int c = 1; c < 4; c++) o = cfma(uel<R, 4>(M, r, c, dag), x[c], o);
      p[idx[r]] = o;
    }
    if (REV) {
#pragma unroll
      for (int c = 0; c < 4; c++) x[c] = l[idx[c]];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        Cx<R> o = cmul(uel<R, 4>(M, r, 0, dag), x[0]);
#pragma unroll
        for (int c = 1; c < 4; c++) o = cfma(uel<R, 4>(M, r, c, dag), x[c], o);
        l[idx[r]] = o;
      }
    }
  }
}

// Anti-diagonal 2x2 on register slot S; FLIP: a pure bit flip (X, CNOT),
// moves only.
template <typename R, int S, bool REV, bool FLIP>
__device__ __forceinline__ void b_anti1(Cx<R> (&p)[NR], Cx<R> (&l)[NR], const BOp& op, const Cx<R>* M) {
  constexpr bool flip = FLIP;
  const Cx<R> a = op.dagger ? conjx(M[1]) : M[0], b = op.dagger ? conjx(M[0]) : M[1];
  const uint32_t rm = op.rmask, rv = op.rval;
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if (j & (1 << S)) continue;
    if ((j & rm) != rv) continue;
    const int j1 = j | (1 << S);
    const Cx<R> x = p[j], y = p[j1];
    p[j] = flip ? y : cmul(a, y);
    p[j1] = flip ? x : cmul(b, x);
    if (REV) {
      const Cx<R> u = l[j], w = l[j1];
      l[j] = flip ? w : cmul(a, w);
      l[j1] = flip ? u : cmul(b, u);
    }
  }
}

template <typename R, int A, int B, bool REV>
__device__ __forceinline__ void b_swap(Cx<R> (&p)[NR], Cx<R> (&l)[NR], const BOp& op) {
  const uint32_t rm = op.rmask, rv = op.rval;
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if (j & ((1 << A) | (1 << B))) continue;
    if ((j & rm) != rv) continue;
    Cx<R> t = p[j | (1 << A)];
    p[j | (1 << A)] = p[j | (1 << B)];
    p[j | (1 << B)] = t;
    if (REV) {
      t = l[j | (1 << A)];
      l[j | (1 << A)] = l[j | (1 << B)];
      l[j | (1 << B)] = t;
    }
  }
}

// x a + y b for real x, y: in single precision the real and imaginary parts
// go through one packed two-lane FP32 multiply and FMA (sm_100 and later),
// rounded as the scalar forms.
template <typename R>
__device__ __forceinline__ Cx<R> rmix2(R x, Cx<R> a, R y, Cx<R> b) {
  if constexpr (sizeof(R) == 4) {
    const float2 r = __ffma2_rn(make_float2(x, x), make_float2(a.re, a.im),
                                __fmul2_rn(make_float2(y, y), make_float2(b.re, b.im)));
    return {r.x, r.y};
  } else {
    return {fma(x, a.re, y * b.re), fma(x, a.im, y * b.im)};
  }
}
// f p as p.re (f.re, f.im) + p.im (-f.im, f.re): one packed multiply and FMA
// in single precision.
template <typename R>
__device__ __forceinline__ Cx<R> pmul(Cx<R> f, Cx<R> v) {
  if constexpr (sizeof(R) == 4) {
    const float2 r = __ffma2_rn(make_float2(v.im, v.im), make_float2(-f.im, f.re),
                                __fmul2_rn(make_float2(v.re, v.re), make_float2(f.re, f.im)));
    return {r.x, r.y};
  } else {
    return cmul(f, v);
  }
}

// Diagonal whose factor depends on at most one register slot S (S < 0: on
// none; the thread's and the tile's fixed bits already picked the entries
// fa / fb).  With GR the gradient term sum Im(conj(lambda) g psi) is added,
// as g.re Im(conj(lambda) psi) + g.im Re(conj(lambda) psi).
template <typename R, int S, bool REV, bool GR>
__device__ __forceinline__ void b_diag_s(Cx<R> (&p)[NR], Cx<R> (&l)[NR], Cx<R> fa, Cx<R> fb, Cx<R> ga, Cx<R> gb,
                                         R& acc) {
#pragma unroll
  for (int j = 0; j < NR; j++) {
    const bool one = S >= 0 && ((j >> (S < 0 ? 0 : S)) & 1);
    if (REV && GR) {
      const Cx<R> g = one ? gb : ga;
      const R cre = fma(l[j].re, p[j].re, l[j].im * p[j].im), cim = fma(l[j].re, p[j].im, -l[j].im * p[j].re);
      acc = fma(g.re, cim, fma(g.im, cre, acc));
    }
    p[j] = cmul(one ? fb : fa, p[j]);
    if (REV) l[j] = cmul(one ? fb : fa, l[j]);
  }
}

template <typename R, bool REV>
__device__ __forceinline__ void b_diag(Cx<R> (&p)[NR], Cx<R> (&l)[NR], const BOp& op, const Cx<R>* M,
                                       const Cx<R>* G, uint32_t tb, uint64_t base, R& acc) {
  uint32_t dbase = 0;
  int s0 = -1, s1 = -1, b0 = 0, b1 = 0;
  for (int i = 0; i < op.k; i++) {
    if (op.rs[i] != 0xFF) {
      if (s0 < 0) {
        s0 = op.rs[i];
        b0 = i;
      } else {
        s1 = op.rs[i];
        b1 = i;
      }
    } else if (op.pos[i] != 0xFF) {
      dbase |= ((tb >> op.pos[i]) & 1u) << i;
    } else {
      dbase |= (uint32_t)((base >> op.gq[i]) & 1ull) << i;
    }
  }
  const uint32_t i1 = s0 >= 0 ? (1u << b0) : 0u, i2 = s1 >= 0 ? (1u << b1) : 0u;
  const bool dag = op.dagger, grad = REV && op.grad;
  if (op.rmask == 0 && s1 < 0) {  // at most one register slot, no register controls
    const Cx<R> fa = dag ? conjx(M[dbase]) : M[dbase], fb = dag ? conjx(M[dbase | i1]) : M[dbase | i1];
    const Cx<R> z = {R(0), R(0)};
    const Cx<R> ga = grad ? G[dbase] : z, gb = grad ? G[dbase | i1] : z;
#define SV_DIAG_S(GR)                                                   \
  switch (s0) {                                                         \
    case -1: b_diag_s<R, -1, REV, GR>(p, l, fa, fb, ga, gb, acc); break; \
    case 0: b_diag_s<R, 0, REV, GR>(p, l, fa, fb, ga, gb, acc); break;   \
    case 1: b_diag_s<R, 1, REV, GR>(p, l, fa, fb, ga, gb, acc); break;   \
    case 2: b_diag_s<R, 2, REV, GR>(p, l, fa, fb, ga, gb, acc); break;   \
    default: b_diag_s<R, 3, REV, GR>(p, l, fa, fb, ga, gb, acc); break;  \
  }
    if (grad) {
      SV_DIAG_S(true)
    } else {
      SV_DIAG_S(false)
    }
#undef SV_DIAG_S
    return;
  }
  Cx<R> f[4], g[4];
  const uint32_t di[4] = {dbase, dbase | i1, dbase | i2, dbase | i1 | i2};
#pragma unroll
  for (int c = 0; c < 4; c++) {
    f[c] = dag ? conjx(M[di[c]]) : M[di[c]];
    g[c] = grad ? G[di[c]] : Cx<R>{R(0), R(0)};
  }
  const int sh0 = s0 >= 0 ? s0 : 0, sh1 = s1 >= 0 ? s1 : 0;
  const uint32_t m0 = s0 >= 0 ? 1u : 0u, m1 = s1 >= 0 ? 1u : 0u;
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if ((j & op.rmask) != op.rval) continue;
    const uint32_t c0 = ((uint32_t)j >> sh0) & m0, c1 = ((uint32_t)j >> sh1) & m1;
    const Cx<R> fj = c1 ? (c0 ? f[3] : f[2]) : (c0 ? f[1] : f[0]);
    if (grad) {
      const Cx<R> gj = c1 ? (c0 ? g[3] : g[2]) : (c0 ? g[1] : g[0]);
      acc += im_cdot(l[j], cmul(gj, p[j]));
    }
    p[j] = cmul(fj, p[j]);
    if (REV) l[j] = cmul(fj, l[j]);
  }
}

// Uncontrolled one-qubit op on register slot S, with the structure of the
// common rotations written out: REAL matrices (RY, H ...) take real products,
// and the gradient term Im <lambda|G|psi> of an X or Y generator (RX, RY) is
// read off the pair directly (GK = 1: X, 2: Y; 0: no gradient).
template <typename R, int S, bool REV, bool REAL, int GK>
__device__ __forceinline__ void b_u1(Cx<R> (&p)[NR], Cx<R> (&l)[NR], const BOp& op, const Cx<R>* M, R& acc) {
  const bool dag = op.dagger;
  const Cx<R> u00 = uel<R, 2>(M, 0, 0, dag), u01 = uel<R, 2>(M, 0, 1, dag);
  const Cx<R> u10 = uel<R, 2>(M, 1, 0, dag), u11 = uel<R, 2>(M, 1, 1, dag);
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if (j & (1 << S)) continue;
    const int j1 = j | (1 << S);
    const Cx<R> a = p[j], b = p[j1];
    if (REV && GK == 1) {  // (X psi) = (b, a)
      acc += im_cdot(l[j], b) + im_cdot(l[j1], a);
    } else if (REV && GK == 2) {  // (Y psi) = (-i b, i a)
      acc += (l[j1].re * a.re + l[j1].im * a.im) - (l[j].re * b.re + l[j].im * b.im);
    }
    if (REAL && sizeof(R) == 4) {  // re and im together: packed two-lane FP32
      p[j] = rmix2(u00.re, a, u01.re, b);
      p[j1] = rmix2(u10.re, a, u11.re, b);
    } else if (REAL) {
      p[j] = {fma(u00.re, a.re, u01.re * b.re), fma(u00.re, a.im, u01.re * b.im)};
      p[j1] = {fma(u10.re, a.re, u11.re * b.re), fma(u10.re, a.im, u11.re * b.im)};
    } else {
      p[j] = cfma(u01, b, cmul(u00, a));
      p[j1] = cfma(u11, b, cmul(u10, a));
    }
    if (REV) {
      const Cx<R> c = l[j], d = l[j1];
      if (REAL && sizeof(R) == 4) {
        l[j] = rmix2(u00.re, c, u01.re, d);
        l[j1] = rmix2(u10.re, c, u11.re, d);
      } else if (REAL) {
        l[j] = {fma(u00.re, c.re, u01.re * d.re), fma(u00.re, c.im, u01.re * d.im)};
        l[j1] = {fma(u10.re, c.re, u11.re * d.re), fma(u10.re, c.im, u11.re * d.im)};
      } else {
        l[j] = cfma(u01, d, cmul(u00, c));
        l[j1] = cfma(u11, d, cmul(u10, c));
      }
    }
  }
}

// Uncontrolled one-qubit diagonal on register slot S (RZ, S, T ...); with GZ
// the gradient term of a Z generator, sum of +-Im(conj(lambda) psi).
template <typename R, int S, bool REV, bool GZ>
__device__ __forceinline__ void b_d1(Cx<R> (&p)[NR], Cx<R> (&l)[NR], const BOp& op, const Cx<R>* M, R& acc) {
  const bool dag = op.dagger;
  const Cx<R> f0 = dag ? conjx(M[0]) : M[0], f1 = dag ? conjx(M[1]) : M[1];
#pragma unroll
  for (int j = 0; j < NR; j++) {
    const bool one = (j >> S) & 1;
    if (REV && GZ) acc += one ? -im_cdot(l[j], p[j]) : im_cdot(l[j], p[j]);
    p[j] = pmul(one ? f1 : f0, p[j]);
    if (REV) l[j] = pmul(one ? f1 : f0, l[j]);
  }
}

// F<R, slot, rest...>(args) for the op's register slot; the last macro
// argument closes the template list and carries the call.
#define SV_SLOT4(F, ...)                    \
  switch (op.rs[0]) {                       \
    case 0: F<R, 0, __VA_ARGS__; break;     \
    case 1: F<R, 1, __VA_ARGS__; break;     \
    case 2: F<R, 2, __VA_ARGS__; break;     \
    default: F<R, 3, __VA_ARGS__; break;    \
  }

template <typename R, bool REV>
__device__ __forceinline__ void b_apply(Cx<R> (&p)[NR], Cx<R> (&l)[NR], const BOp& op, const Cx<R>* M,
                                        const Cx<R>* G, uint32_t tb, uint64_t base, R& acc) {
  const bool plain = op.rmask == 0 && op.rs[0] != 0xFF;  // uncontrolled, on a register slot
  if (plain && op.k == 1 && (op.kind == OPK_DENSE || op.kind == OPK_REAL)) {
    const bool real = op.flags & OPF_REALM;
    const int gk = !(REV && op.grad) ? 0 : (op.flags & OPF_GX) ? 1 : (op.flags & OPF_GY) ? 2 : 3;
    if (gk != 3) {
      if (real && gk == 2) {
        SV_SLOT4(b_u1, REV, true, 2>(p, l, op, M, acc))
      } else if (real && gk == 0) {
        SV_SLOT4(b_u1, REV, true, 0>(p, l, op, M, acc))
      } else if (gk == 1) {
        SV_SLOT4(b_u1, REV, false, 1>(p, l, op, M, acc))
      } else if (gk == 0) {
        SV_SLOT4(b_u1, REV, false, 0>(p, l, op, M, acc))
      } else {
        SV_SLOT4(b_u1, REV, false, 2>(p, l, op, M, acc))
      }
      return;
    }
  }
  if (plain && op.k == 1 && op.kind == OPK_DIAG) {
    const bool gz = REV && op.grad && (op.flags & OPF_GZ);
    if (gz || !(REV && op.grad)) {
      if (gz) {
        SV_SLOT4(b_d1, REV, true>(p, l, op, M, acc))
      } else {
        SV_SLOT4(b_d1, REV, false>(p, l, op, M, acc))
      }
      return;
    }
  }
  switch (op.kind) {
    case OPK_DENSE:
    case OPK_REAL:
      if (op.k == 1) {
        switch (op.rs[0]) {
          case 0: b_dense1<R, 0, REV>(p, l, op, M, G, acc); break;
          case 1: b_dense1<R, 1, REV>(p, l, op, M, G, acc); break;
          case 2: b_dense1<R, 2, REV>(p, l, op, M, G, acc); break;
          default: b_dense1<R, 3, REV>(p, l, op, M, G, acc); break;
        }
      } else {
        switch (op.rs[0] * 4 + op.rs[1]) {
          case 1: b_dense2<R, 0, 1, REV>(p, l, op, M, G, acc); break;
          case 2: b_dense2<R, 0, 2, REV>(p, l, op, M, G, acc); break;
          case 3: b_dense2<R, 0, 3, REV>(p, l, op, M, G, acc); break;
          case 4: b_dense2<R, 1, 0, REV>(p, l, op, M, G, acc); break;
          case 6: b_dense2<R, 1, 2, REV>(p, l, op, M, G, acc); break;
          case 7: b_dense2<R, 1, 3, REV>(p, l, op, M, G, acc); break;
          case 8: b_dense2<R, 2, 0, REV>(p, l, op, M, G, acc); break;
          case 9: b_dense2<R, 2, 1, REV>(p, l, op, M, G, acc); break;
          case 11: b_dense2<R, 2, 3, REV>(p, l, op, M, G, acc); break;
          case 12: b_dense2<R, 3, 0, REV>(p, l, op, M, G, acc); break;
          case 13: b_dense2<R, 3, 1, REV>(p, l, op, M, G, acc); break;
          default: b_dense2<R, 3, 2, REV>(p, l, op, M, G, acc); break;
        }
      }
      break;
    case OPK_ANTIDIAG:
      if (op.flags & OPF_FLIP) {
        SV_SLOT4(b_anti1, REV, true>(p, l, op, M))
      } else {
        SV_SLOT4(b_anti1, REV, false>(p, l, op, M))
      }
      break;
    case OPK_SWAP: {
      const int a = op.rs[0] < op.rs[1] ? op.rs[0] : op.rs[1], b = op.rs[0] < op.rs[1] ? op.rs[1] : op.rs[0];
      switch (a * 4 + b) {
        case 1: b_swap<R, 0, 1, REV>(p, l, op); break;
        case 2: b_swap<R, 0, 2, REV>(p, l, op); break;
        case 3: b_swap<R, 0, 3, REV>(p, l, op); break;
        case 6: b_swap<R, 1, 2, REV>(p, l, op); break;
        case 7: b_swap<R, 1, 3, REV>(p, l, op); break;
        default: b_swap<R, 2, 3, REV>(p, l, op); break;
      }
      break;
    }
    case OPK_DIAG: b_diag<R, REV>(p, l, op, M, G, tb, base, acc); break;
    default: break;
  }
}

template <typename R, bool REV>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) k_batch_sweep(Cx<R>* __restrict__ psi, Cx<R>* __restrict__ lam,
                                                     const Cx<R>* __restrict__ table, double* __restrict__ gscratch,
                                                     const __grid_constant__ BatchProgram<R> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchHeader& h = P.h;
  const int tsz = 1 << h.m;
  Cx<R>* sp = reinterpret_cast<Cx<R>*>(smem_raw);
  Cx<R>* sl = sp + (REV ? tsz : 0);
  uint64_t* hi_off = reinterpret_cast<uint64_t*>(sp + (REV ? 2 * tsz : tsz));
  // this state's coefficients (table rows and constant matrices) and the
  // generators, copied once per CTA
  Cx<R>* scoef = reinterpret_cast<Cx<R>*>(hi_off + (1 << (h.m - h.L)));
  __shared__ double gacc[kBatchGacc][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kBatchGacc * 8; i += blockDim.x) gacc[i / 8][i % 8] = 0.0;
  const int bidx = blockIdx.y;
  Cx<R>* ps = psi + ((uint64_t)bidx << h.n);
  Cx<R>* ls = REV ? lam + ((uint64_t)bidx << h.n) : nullptr;
  constexpr int A = 16 / sizeof(Cx<R>);
  const int nvec = tsz / A;
  const uint64_t ntiles = 1ull << (h.n - h.m);
  const int nhi = 1 << (h.m - h.L);
  for (int c = threadIdx.x; c < nhi; c += blockDim.x) hi_off[c] = local_offset((uint32_t)c << h.L, h);
  for (int o = warp; o < h.nops; o += (int)(blockDim.x >> 5)) {
    const BOp& op = P.ops[o];
    const int dd = 1 << op.k;
    const int mc = op.kind == OPK_DIAG ? dd : op.kind == OPK_ANTIDIAG ? 2 : op.kind == OPK_SWAP ? 0 : dd * dd;
    const int gc = op.grad ? (op.kind == OPK_DIAG ? dd : dd * dd) : 0;
    const Cx<R>* src = op.table ? table + ((uint64_t)op.coef * h.batch + bidx) * kTableStride : P.pool + op.coef;
    for (int e = lane; e < mc + gc; e += 32) scoef[op.soff + e] = e < mc ? src[e] : P.pool[op.gen + (e - mc)];
  }
  const uint32_t lowmask = (1u << h.L) - 1u;
  __syncthreads();
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    uint64_t base = tile;
    for (int i = 0; i < h.m; i++) base = ins0_64(base, h.tq[i]);
    // asynchronous 16-byte copies, all in flight before one wait
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
      const uint32_t l = (uint32_t)(v * A);
      const uint64_t off = base + (hi_off[l >> h.L] | (l & lowmask));
      cp_async16(sp + sw<R>(l), ps + off);
      if (REV) cp_async16(sl + sw<R>(l), ls + off);
    }
    cp_async_commit_wait_all();
    __syncthreads();
    for (int ph_i = 0; ph_i < h.nphases; ph_i++) {
      const Phase& ph = P.ph[ph_i];
      if (ph.kind == PH_REG) {
        const bool active = threadIdx.x < (1u << ph.ntpos);
        if ((threadIdx.x & ~31u) < (1u << ph.ntpos)) {  // the warp holds at least one group
          // thread bits: the thread index with zeros inserted at the register
          // positions (ascending); the swizzle is linear over XOR, so each
          // register slot is one XOR away from one formed before it
          uint32_t tb = threadIdx.x;
#pragma unroll
          for (int i = 0; i < kRegQ; i++) tb = ins0(tb, ph.rp[i]);
          auto slots = [&](uint32_t (&off)[NR]) {  // formed again for the store: no registers held across ops
            off[0] = sw<R>(tb);
#pragma unroll
            for (int j = 1; j < NR; j++) {
              const int low = j & -j;
              const int i = low == 1 ? 0 : low == 2 ? 1 : low == 4 ? 2 : 3;
              off[j] = off[j ^ low] ^ sw<R>(1u << ph.rp[i]);
            }
          };
          Cx<R> p[NR], l[NR];
          if (active) {
            uint32_t off[NR];
            slots(off);
            if (sizeof(Cx<R>) == 8 && ph.rp[0] == 0) {  // pairs (j, j+1) share a 16-byte granule
#pragma unroll
              for (int j = 0; j < NR; j += 2) {
                const float4 a = *reinterpret_cast<const float4*>(sp + off[j]);
                p[j] = Cx<R>{(R)a.x, (R)a.y};
                p[j + 1] = Cx<R>{(R)a.z, (R)a.w};
                if (REV) {
                  const float4 b = *reinterpret_cast<const float4*>(sl + off[j]);
                  l[j] = Cx<R>{(R)b.x, (R)b.y};
                  l[j + 1] = Cx<R>{(R)b.z, (R)b.w};
                }
              }
            } else {
#pragma unroll
              for (int j = 0; j < NR; j++) {
                p[j] = sp[off[j]];
                if (REV) l[j] = sl[off[j]];
              }
            }
          }
          for (int o = ph.first; o < ph.first + ph.nops; o++) {
            const BOp& op = P.ops[o];
            R acc = R(0);
            if (active && (base & op.xmask) == op.xval && (tb & op.tmask) == op.tval) {
              const Cx<R>* M = scoef + op.soff;
              const int dd = 1 << op.k;
              const Cx<R>* G = M + (op.kind == OPK_DIAG ? dd : dd * dd);
              b_apply<R, REV>(p, l, op, M, G, tb, base, acc);
            }
            if (REV && op.grad) {  // warp sum in the state's precision, then double
              R w = acc;
#pragma unroll
              for (int s2 = 16; s2 > 0; s2 >>= 1) w += __shfl_xor_sync(0xffffffffu, w, s2);
              if (lane == 0) gacc[op.gacc][warp] += (double)w;
            }
          }
          if (active) {
            uint32_t off[NR];
            slots(off);
            if (sizeof(Cx<R>) == 8 && ph.rp[0] == 0) {
#pragma unroll
              for (int j = 0; j < NR; j += 2) {
                *reinterpret_cast<float4*>(sp + off[j]) =
                    make_float4((float)p[j].re, (float)p[j].im, (float)p[j + 1].re, (float)p[j + 1].im);
                if (REV)
                  *reinterpret_cast<float4*>(sl + off[j]) =
                      make_float4((float)l[j].re, (float)l[j].im, (float)l[j + 1].re, (float)l[j + 1].im);
              }
            } else {
#pragma unroll
              for (int j = 0; j < NR; j++) {
                sp[off[j]] = p[j];
                if (REV) sl[off[j]] = l[j];
              }
            }
          }
        }
      } else {
        // tiles too small for register groups (m < 4): the op group by group
        // in shared memory, through the same swizzle
        const BOp& op = P.ops[ph.first];
        if ((base & op.xmask) == op.xval) {
          const Cx<R>* M = scoef + op.soff;
          const int dd = 1 << op.k;
          const Cx<R>* G = M + (op.kind == OPK_DIAG ? dd : dd * dd);
          R acc = R(0);
          switch (op.kind) {
            case OPK_DENSE:
            case OPK_REAL:
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
        } else if (REV && op.grad) {
          // nothing to add, but keep the warp reduction uniform
        }
      }
      __syncthreads();
    }
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
      const uint32_t l = (uint32_t)(v * A);
      const uint64_t off = base + (hi_off[l >> h.L] | (l & lowmask));
      *reinterpret_cast<uint4*>(ps + off) = *reinterpret_cast<const uint4*>(sp + sw<R>(l));
      if (REV) *reinterpret_cast<uint4*>(ls + off) = *reinterpret_cast<const uint4*>(sl + sw<R>(l));
    }
    __syncthreads();
  }
  if (REV) {
    for (int o = threadIdx.x; o < h.nops; o += blockDim.x) {
      const BOp& op = P.ops[o];
      if (!op.grad) continue;
      double s2 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) s2 += gacc[op.gacc][w];
      gscratch[((uint64_t)bidx * h.ngrad_total + op.gidx) * gridDim.x + blockIdx.x] = s2;
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
                               const BatchProgram<R>& prog, bool reverse, cudaStream_t stream) {
  const int smem = ((int)sizeof(Cx<R>) << prog.h.m << (reverse ? 1 : 0)) + (8 << (prog.h.m - prog.h.L)) +
                   (int)sizeof(Cx<R>) * prog.h.scoef;
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
    kernel<<<grid, 256, smem, stream>>>(psi, lam, table, gscratch, prog);
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
                                             bool, cudaStream_t);                                                 \
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
