// sv_batch_ops.cuh -- what a batched adjoint pass does to one tile of psi and
// lambda: the shared-memory ops, the register ops (every register slot a
// compile-time constant) with their gradient terms, and the tile loop of a
// pass (gather, phases, scatter, per-CTA gradient partials).  Included by the
// library's interpreting kernel (sv_adjoint.cu) and by the kernels compiled at
// run time from one batched program (sv_jit_batch.cpp), which call the same
// functions with every op field a constant, so both paths round alike.
// Device code only, no host headers.
#pragma once

#include "sv_batch_layout.h"
#include "sv_pass_ops.cuh"

namespace sv {

template <typename R>
__device__ __forceinline__ Cx<R> conjx(Cx<R> a) {
  return {a.re, -a.im};
}
// Im(conj(l) * g) = l.re g.im - l.im g.re, its rounding fixed in the source
// (one product, one fused multiply-add) so that every compilation of the
// gradient terms rounds alike.
template <typename R>
__device__ __forceinline__ R im_cdot(Cx<R> l, Cx<R> g) {
  return fma(l.re, g.im, -(l.im * g.re));
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

// Shared-memory slot of local amplitude l (the XOR swizzle of the
// single-state sweep).
template <typename R>
__device__ __forceinline__ uint32_t sw(uint32_t l) {
  return phys<R>(l);
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
      acc += fma(l[j1].re, a.re, l[j1].im * a.im) - fma(l[j].re, b.re, l[j].im * b.im);
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
#define SV_BSLOT4(F, ...)                    \
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
        SV_BSLOT4(b_u1, REV, true, 2>(p, l, op, M, acc))
      } else if (real && gk == 0) {
        SV_BSLOT4(b_u1, REV, true, 0>(p, l, op, M, acc))
      } else if (gk == 1) {
        SV_BSLOT4(b_u1, REV, false, 1>(p, l, op, M, acc))
      } else if (gk == 0) {
        SV_BSLOT4(b_u1, REV, false, 0>(p, l, op, M, acc))
      } else {
        SV_BSLOT4(b_u1, REV, false, 2>(p, l, op, M, acc))
      }
      return;
    }
  }
  if (plain && op.k == 1 && op.kind == OPK_DIAG) {
    const bool gz = REV && op.grad && (op.flags & OPF_GZ);
    if (gz || !(REV && op.grad)) {
      if (gz) {
        SV_BSLOT4(b_d1, REV, true>(p, l, op, M, acc))
      } else {
        SV_BSLOT4(b_d1, REV, false>(p, l, op, M, acc))
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
        SV_BSLOT4(b_anti1, REV, true>(p, l, op, M))
      } else {
        SV_BSLOT4(b_anti1, REV, false>(p, l, op, M))
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

// The tile loop of a batched pass (grid.y the state, grid.x the CTAs of one
// state, 256 threads): the op coefficients of this state (table rows and
// constant matrices) and the generators are copied to shared memory once per
// CTA; each tile of psi (and, in reverse, lambda) is gathered with 16-byte
// asynchronous copies, runner(sp, sl, tsz, scoef, base, gacc, warp, lane) runs
// the program's phases on it (a barrier after each), and the tile is written
// back; per-CTA gradient partials go to gscratch.
template <typename R, bool REV, class Runner>
__device__ __forceinline__ void batch_sweep_body(Cx<R>* __restrict__ psi, Cx<R>* __restrict__ lam,
                                                 const Cx<R>* __restrict__ table, double* __restrict__ gscratch,
                                                 const BatchProgram<R>& P, const Runner& runner) {
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
    runner(sp, sl, tsz, scoef, base, gacc, warp, lane);
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

// One register phase of a batched pass: each active thread loads the 16
// amplitudes of psi (and lambda) at the phase's register positions rp[] with
// the thread index deposited into the other local bits, ops(p, l, tb, active)
// applies the phase's ops to them, and the thread stores them back.  Threads
// of warps beyond the phase's groups skip it.
template <typename R, bool REV, class Ops>
__device__ __forceinline__ void batch_reg_phase(const Phase& ph, Cx<R>* sp, Cx<R>* sl, const Ops& ops) {
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
    ops(p, l, tb, active);
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
}

// A gradient op's term over the warp: summed in the state's precision, then
// added in double to the op's accumulator (one slot per warp).
template <typename R>
__device__ __forceinline__ void batch_grad_add(R acc, double* row, int warp, int lane) {
  R w = acc;
#pragma unroll
  for (int s2 = 16; s2 > 0; s2 >>= 1) w += __shfl_xor_sync(0xffffffffu, w, s2);
  if (lane == 0) row[warp] += (double)w;
}

// One op of a register phase on the thread's registers (when the op's
// controls on the tile's and the thread's fixed bits hold), then, for a
// gradient op, the warp's sum of its term in the state's precision added in
// double to the op's accumulator.
template <typename R, bool REV>
__device__ __forceinline__ void batch_reg_op(const BOp& op, Cx<R> (&p)[NR], Cx<R> (&l)[NR], uint32_t tb, bool active,
                                             const Cx<R>* scoef, uint64_t base, double (*gacc)[8], int warp,
                                             int lane) {
  R acc = R(0);
  if (active && (base & op.xmask) == op.xval && (tb & op.tmask) == op.tval) {
    const Cx<R>* M = scoef + op.soff;
    const int dd = 1 << op.k;
    const Cx<R>* G = M + (op.kind == OPK_DIAG ? dd : dd * dd);
    b_apply<R, REV>(p, l, op, M, G, tb, base, acc);
  }
  if (REV && op.grad) batch_grad_add<R>(acc, gacc[op.gacc], warp, lane);
}

// One op of a shared-memory phase (tiles too small for register groups):
// the op group by group in shared memory, through the same swizzle.
template <typename R, bool REV>
__device__ __forceinline__ void batch_smem_op(const BOp& op, Cx<R>* sp, Cx<R>* sl, int tsz, const Cx<R>* scoef,
                                              uint64_t base, double (*gacc)[8], int warp, int lane) {
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
  }
}

// Runs a batched program's phases on one tile by interpreting them.
template <typename R, bool REV>
struct BatchInterp {
  const BatchProgram<R>& P;
  __device__ __forceinline__ void operator()(Cx<R>* sp, Cx<R>* sl, int tsz, const Cx<R>* scoef, uint64_t base,
                                             double (*gacc)[8], int warp, int lane) const {
    const BatchHeader& h = P.h;
    for (int ph_i = 0; ph_i < h.nphases; ph_i++) {
      const Phase& ph = P.ph[ph_i];
      if (ph.kind == PH_REG) {
        batch_reg_phase<R, REV>(ph, sp, sl, [&](Cx<R>(&p)[NR], Cx<R>(&l)[NR], uint32_t tb, bool active) {
          for (int o = ph.first; o < ph.first + ph.nops; o++)
            batch_reg_op<R, REV>(P.ops[o], p, l, tb, active, scoef, base, gacc, warp, lane);
        });
      } else {
        batch_smem_op<R, REV>(P.ops[ph.first], sp, sl, tsz, scoef, base, gacc, warp, lane);
      }
      __syncthreads();
    }
  }
};

}  // namespace sv
