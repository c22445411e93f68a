// sv_pass_ops.cuh -- what a pass does to one tile in shared memory: the
// register ops (every register slot a compile-time constant), the register
// loads and stores of a phase, the shared-memory ops of wide gates and the
// direct store of a last register phase to the state.  Included by the
// library's interpreting pass kernel (sv_sweep.cu), by the pass kernels
// compiled at run time from one program (sv_jit.cpp), which call the same
// functions with constant arguments, so both paths round alike, and by the
// batched adjoint sweeps (sv_batch_ops.cuh: the complex product and the bit
// helpers).  Device code only, no host headers.
#pragma once

#include "sv_prog_layout.h"

namespace sv {

template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {  // rounding fixed: one product, one fma per part
  return {fma(a.re, b.re, -(a.im * b.im)), fma(a.re, b.im, a.im * b.re)};
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

// Shared-memory slot of local amplitude l: the 16-byte granule index has its
// low three bits XORed with the next three (bit 0 of a complex64 index, the
// amplitude inside its granule, is left alone).
template <typename R>
__device__ __forceinline__ uint32_t phys(uint32_t l) {
  if constexpr (sizeof(Cx<R>) == 8)
    return l ^ ((l >> 3) & 14u);
  else
    return l ^ ((l >> 3) & 7u);
}

// ---------------------------------------------------------------- register ops
//
// A register phase gives each thread NR = 2^RQ amplitudes that differ only on
// the phase's RQ register tile qubits (RQ = 4 or 5).  Every op below is fully
// unrolled over the NR registers; its register slots are template arguments
// picked by a switch, so every register index is a compile-time constant.

// Controlled (or real) 2x2 matrix on register slot S; the register-slot part
// of the controls is a per-pair predicate applied with selects.
template <typename R, int RQ, int S, bool REAL>
__device__ __forceinline__ void r_dense1(Cx<R> (&v)[1 << RQ], const Cx<R>* cf, uint32_t rmask, uint32_t rval) {
  constexpr int NR = 1 << RQ;
  const Cx<R> u00 = cf[0], u01 = cf[1], u10 = cf[2], u11 = cf[3];
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if (j & (1 << S)) continue;
    const int j1 = j | (1 << S);
    const bool on = (j & rmask) == rval;
    const Cx<R> a = v[j], b = v[j1];
    Cx<R> o0, o1;
    if (REAL) {
      o0 = {fma(u00.re, a.re, u01.re * b.re), fma(u00.re, a.im, u01.re * b.im)};
      o1 = {fma(u10.re, a.re, u11.re * b.re), fma(u10.re, a.im, u11.re * b.im)};
    } else {
      o0 = cfma(u01, b, cmul(u00, a));
      o1 = cfma(u11, b, cmul(u10, a));
    }
    v[j] = on ? o0 : a;
    v[j1] = on ? o1 : b;
  }
}

// Uncontrolled 2x2 complex matrix on register slot S.
template <typename R, int RQ, int S>
__device__ __forceinline__ void r_u1(Cx<R> (&v)[1 << RQ], const Cx<R>* cf) {
  constexpr int NR = 1 << RQ;
  const Cx<R> u00 = cf[0], u01 = cf[1], u10 = cf[2], u11 = cf[3];
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if (j & (1 << S)) continue;
    const int j1 = j | (1 << S);
    const Cx<R> a = v[j], b = v[j1];
    v[j] = cfma(u01, b, cmul(u00, a));
    v[j1] = cfma(u11, b, cmul(u10, a));
  }
}

// Real rotation [[C, -S], [S, C]] on register slot S.
//  - complex64 (issue-bound): three in-place shears a -= t b; b += s a;
//    a -= t b with coef = (t, s) = (tan(alpha/2), sin(alpha)); no
//    temporaries, one packed FMA per shear.
//  - complex128 (FP64-pipe-bound): two FMAs per component in scaled form,
//    the scale carried by a phase table: coef.re = t and, with COT clear,
//    (a, b) -> (a - t b, b + t a) (scale C, t = S/C); with COT set,
//    (a, b) -> (t a - b, a + t b) (scale S, t = C/S).
// a += c * b for the real and imaginary parts at once: one packed two-lane
// FP32 FMA (sm_100 and later), rounded exactly as two scalar FMAs.
__device__ __forceinline__ void shear2(Cx<float>& a, float2 c, const Cx<float>& b) {
  const float2 r = __ffma2_rn(c, make_float2(b.re, b.im), make_float2(a.re, a.im));
  a.re = r.x;
  a.im = r.y;
}

template <typename R, int RQ, int S, bool COT>
__device__ __forceinline__ void r_rot(Cx<R> (&v)[1 << RQ], Cx<R> ts) {
  constexpr int NR = 1 << RQ;
  const R t = ts.re, sn = ts.im;
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if (j & (1 << S)) continue;
    const int j1 = j | (1 << S);
    if constexpr (sizeof(R) == 4) {
      const float2 mt = make_float2(-t, -t), ms = make_float2(sn, sn);
      shear2(v[j], mt, v[j1]);
      shear2(v[j1], ms, v[j]);
      shear2(v[j], mt, v[j1]);
    } else {
      const Cx<R> a = v[j], b = v[j1];
      if (COT) {
        v[j] = {fma(t, a.re, -b.re), fma(t, a.im, -b.im)};
        v[j1] = {fma(t, b.re, a.re), fma(t, b.im, a.im)};
      } else {
        v[j] = {fma(-t, b.re, a.re), fma(-t, b.im, a.im)};
        v[j1] = {fma(t, a.re, b.re), fma(t, a.im, b.im)};
      }
    }
  }
}

template <typename R, int RQ, int S>
__device__ __forceinline__ void r_rot_slot(Cx<R> (&v)[1 << RQ], const Cx<R>* cf, uint32_t cot) {
  if (sizeof(R) == 8 && ((cot >> S) & 1u))
    r_rot<R, RQ, S, true>(v, cf[S]);
  else
    r_rot<R, RQ, S, false>(v, cf[S]);
}

// Anti-diagonal 2x2 on register slot S: a pure bit flip (X, CNOT) when FLIP,
// else out0 = a01 v1, out1 = a10 v0 (Y ...); register-slot controls by select.
template <typename R, int RQ, int S, bool FLIP>
__device__ __forceinline__ void r_anti1(Cx<R> (&v)[1 << RQ], const Cx<R>* cf, uint32_t rmask, uint32_t rval) {
  constexpr int NR = 1 << RQ;
  Cx<R> a01 = {R(1), R(0)}, a10 = {R(1), R(0)};
  if (!FLIP) {
    a01 = cf[0];
    a10 = cf[1];
  }
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if (j & (1 << S)) continue;
    const int j1 = j | (1 << S);
    const bool on = (j & rmask) == rval;
    const Cx<R> a = v[j], b = v[j1];
    const Cx<R> o0 = FLIP ? b : cmul(a01, b), o1 = FLIP ? a : cmul(a10, a);
    v[j] = on ? o0 : a;
    v[j1] = on ? o1 : b;
  }
}

template <typename R, int RQ, int A, int B>
__device__ __forceinline__ void r_dense2(Cx<R> (&v)[1 << RQ], const Cx<R>* cf, uint32_t rmask, uint32_t rval) {
  constexpr int NR = 1 << RQ;
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if (j & ((1 << A) | (1 << B))) continue;
    if ((j & rmask) != rval) continue;
    const int i0 = j, i1 = j | (1 << A), i2 = j | (1 << B), i3 = j | (1 << A) | (1 << B);
    const Cx<R> x0 = v[i0], x1 = v[i1], x2 = v[i2], x3 = v[i3];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      Cx<R> acc = cmul(cf[r * 4 + 0], x0);
      acc = cfma(cf[r * 4 + 1], x1, acc);
      acc = cfma(cf[r * 4 + 2], x2, acc);
      acc = cfma(cf[r * 4 + 3], x3, acc);
      v[r == 0 ? i0 : r == 1 ? i1 : r == 2 ? i2 : i3] = acc;
    }
  }
}

template <typename R, int RQ, int A, int B>
__device__ __forceinline__ void r_swap(Cx<R> (&v)[1 << RQ], uint32_t rmask, uint32_t rval) {
  constexpr int NR = 1 << RQ;
#pragma unroll
  for (int j = 0; j < NR; j++) {
    if (j & ((1 << A) | (1 << B))) continue;
    if ((j & rmask) != rval) continue;
    const Cx<R> t = v[j | (1 << A)];
    v[j | (1 << A)] = v[j | (1 << B)];
    v[j | (1 << B)] = t;
  }
}

template <typename R, int RQ>
__device__ __forceinline__ void apply_neg(Cx<R> (&v)[1 << RQ], uint32_t neg) {
#pragma unroll
  for (int j = 0; j < (1 << RQ); j++) {
    if ((neg >> j) & 1u) {
      v[j].re = -v[j].re;
      v[j].im = -v[j].im;
    }
  }
}

// Diagonal op with k <= 2 matrix bits, each held by a register slot, by the
// thread index, or fixed for the tile.
template <typename R, int RQ>
__device__ __forceinline__ void r_diag(Cx<R> (&v)[1 << RQ], const DevOp& op, const Cx<R>* cf, uint32_t tb,
                                       uint64_t base) {
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
  const Cx<R> f0 = cf[dbase];
  const Cx<R> f1 = s0 >= 0 ? cf[dbase | (1u << b0)] : f0;
  const Cx<R> f2 = s1 >= 0 ? cf[dbase | (1u << b1)] : f0;
  const Cx<R> f3 = s1 >= 0 ? cf[dbase | (1u << b0) | (1u << b1)] : f1;
  const int sh0 = s0 >= 0 ? s0 : 0, sh1 = s1 >= 0 ? s1 : 0;
  const uint32_t m0 = s0 >= 0 ? 1u : 0u, m1 = s1 >= 0 ? 1u : 0u;
#pragma unroll
  for (int j = 0; j < (1 << RQ); j++) {
    if ((j & op.rmask) != op.rval) continue;
    const uint32_t c0 = ((uint32_t)j >> sh0) & m0, c1 = ((uint32_t)j >> sh1) & m1;
    const Cx<R> f = c1 ? (c0 ? f3 : f2) : (c0 ? f1 : f0);
    v[j] = cmul(f, v[j]);
  }
}

// v[j] *= T0[j] over the thread's 2^RQ amplitudes (one variant of a phase
// table), with one temporary: everything else in place.
template <typename R, int RQ>
__device__ __forceinline__ void r_phase_table(Cx<R> (&v)[1 << RQ], const Cx<R>* T0) {
  auto mul = [](Cx<R>& x, R tr, R ti) {
    const R t = x.im * ti;
    x.im = fma(x.re, ti, x.im * tr);
    x.re = fma(x.re, tr, -t);
  };
  if constexpr (sizeof(R) == 4) {  // pairs of entries per 16-byte load
#pragma unroll
    for (int j = 0; j < (1 << RQ); j += 2) {
      const float4 w = *reinterpret_cast<const float4*>(T0 + j);
      mul(v[j], (R)w.x, (R)w.y);
      mul(v[j + 1], (R)w.z, (R)w.w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < (1 << RQ); j++) mul(v[j], T0[j].re, T0[j].im);
  }
}

// Shared-memory slots of a thread's register combinations.  The swizzle is
// linear over XOR and the thread bits tb are disjoint from the register bits,
// so phys(tb | bits(j)) = phys(tb) ^ (XOR of phys(m[i]) over the set bits i of
// j): each slot is one XOR away from a slot computed before it.  With STEP = 2
// only even j are formed (pairs sharing a 16-byte granule).
template <typename R, int RQ, int STEP>
__device__ __forceinline__ void reg_slots(uint32_t (&off)[(1 << RQ) / STEP], uint32_t tb, const uint32_t (&m)[RQ]) {
  off[0] = phys<R>(tb);
#pragma unroll
  for (int j = STEP; j < (1 << RQ); j += STEP) {
    const int low = j & -j;  // lowest set bit of j
    const int i = low == 1 ? 0 : low == 2 ? 1 : low == 4 ? 2 : low == 8 ? 3 : 4;
    off[j / STEP] = off[(j ^ low) / STEP] ^ phys<R>(m[i]);
  }
}

// Register loads and stores through any layout that is linear over XOR, as
// the kernels compiled from one program use between two register phases:
// s0 is the slot of the thread's base index tb and ms[i] the slot of
// register bit i alone, so combination j sits at s0 ^ (XOR of ms[i] over the
// set bits i of j).  PAIRS: register bit 0 is local bit 0 and the layout
// keeps pairs (j, j+1) in one 16-byte granule, in order.
template <int RQ, int STEP>
__device__ __forceinline__ void reg_slots_at(uint32_t (&off)[(1 << RQ) / STEP], uint32_t s0,
                                             const uint32_t (&ms)[RQ]) {
  off[0] = s0;
#pragma unroll
  for (int j = STEP; j < (1 << RQ); j += STEP) {
    const int low = j & -j;
    const int i = low == 1 ? 0 : low == 2 ? 1 : low == 4 ? 2 : low == 8 ? 3 : 4;
    off[j / STEP] = off[(j ^ low) / STEP] ^ ms[i];
  }
}

template <typename R, int RQ, bool PAIRS>
__device__ __forceinline__ void reg_load_at(Cx<R> (&v)[1 << RQ], const Cx<R>* s, uint32_t s0,
                                            const uint32_t (&ms)[RQ]) {
  if constexpr (PAIRS && sizeof(Cx<R>) == 8) {
    uint32_t off[(1 << RQ) / 2];
    reg_slots_at<RQ, 2>(off, s0, ms);
#pragma unroll
    for (int j = 0; j < (1 << RQ); j += 2) {
      const float4 w = *reinterpret_cast<const float4*>(s + off[j / 2]);
      v[j] = Cx<R>{(R)w.x, (R)w.y};
      v[j + 1] = Cx<R>{(R)w.z, (R)w.w};
    }
  } else {
    uint32_t off[1 << RQ];
    reg_slots_at<RQ, 1>(off, s0, ms);
#pragma unroll
    for (int j = 0; j < (1 << RQ); j++) v[j] = s[off[j]];
  }
}

template <typename R, int RQ, bool PAIRS>
__device__ __forceinline__ void reg_store_at(const Cx<R> (&v)[1 << RQ], Cx<R>* s, uint32_t s0,
                                             const uint32_t (&ms)[RQ]) {
  if constexpr (PAIRS && sizeof(Cx<R>) == 8) {
    uint32_t off[(1 << RQ) / 2];
    reg_slots_at<RQ, 2>(off, s0, ms);
#pragma unroll
    for (int j = 0; j < (1 << RQ); j += 2)
      *reinterpret_cast<float4*>(s + off[j / 2]) =
          make_float4((float)v[j].re, (float)v[j].im, (float)v[j + 1].re, (float)v[j + 1].im);
  } else {
    uint32_t off[1 << RQ];
    reg_slots_at<RQ, 1>(off, s0, ms);
#pragma unroll
    for (int j = 0; j < (1 << RQ); j++) s[off[j]] = v[j];
  }
}

template <typename R, int RQ>
__device__ __forceinline__ void reg_load(Cx<R> (&v)[1 << RQ], const Cx<R>* s, uint32_t tb, const uint32_t (&m)[RQ]) {
  if (sizeof(Cx<R>) == 8 && m[0] == 1u) {  // pairs (j, j+1) share a 16-byte granule
    uint32_t off[(1 << RQ) / 2];
    reg_slots<R, RQ, 2>(off, tb, m);
#pragma unroll
    for (int j = 0; j < (1 << RQ); j += 2) {
      const float4 w = *reinterpret_cast<const float4*>(s + off[j / 2]);
      v[j] = Cx<R>{(R)w.x, (R)w.y};
      v[j + 1] = Cx<R>{(R)w.z, (R)w.w};
    }
  } else {
    uint32_t off[1 << RQ];
    reg_slots<R, RQ, 1>(off, tb, m);
#pragma unroll
    for (int j = 0; j < (1 << RQ); j++) v[j] = s[off[j]];
  }
}

template <typename R, int RQ>
__device__ __forceinline__ void reg_store(const Cx<R> (&v)[1 << RQ], Cx<R>* s, uint32_t tb,
                                          const uint32_t (&m)[RQ]) {
  if (sizeof(Cx<R>) == 8 && m[0] == 1u) {
    uint32_t off[(1 << RQ) / 2];
    reg_slots<R, RQ, 2>(off, tb, m);
#pragma unroll
    for (int j = 0; j < (1 << RQ); j += 2)
      *reinterpret_cast<float4*>(s + off[j / 2]) =
          make_float4((float)v[j].re, (float)v[j].im, (float)v[j + 1].re, (float)v[j + 1].im);
  } else {
    uint32_t off[1 << RQ];
    reg_slots<R, RQ, 1>(off, tb, m);
#pragma unroll
    for (int j = 0; j < (1 << RQ); j++) s[off[j]] = v[j];
  }
}

// ---------------------------------------------------------------- shared-memory ops
// The threads that share one tile: the whole CTA (bar == 0, __syncthreads),
// or one group of a CTA that works on several tiles at once (named barrier `bar` over
// `nthr` threads, a multiple of 32).  tid is the thread's index in the group.
struct Grp {
  uint32_t tid, nthr, bar;
};
__device__ __forceinline__ void grp_sync(const Grp& g) {
  if (g.bar == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;\n" ::"r"(g.bar), "r"(g.nthr) : "memory");
}


template <typename R, int K>
__device__ __forceinline__ void s_denseK(Cx<R>* s, int tsz, const DevOp& op, const Cx<R>* cf, const Grp& gr) {
  constexpr int D = 1 << K;
  uint32_t bit[K];
#pragma unroll
  for (int i = 0; i < K; i++) bit[i] = 1u << op.pos[i];
  for (uint32_t g = gr.tid; g < (uint32_t)(tsz >> K); g += gr.nthr) {
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
      v[j] = s[phys<R>(x)];
    }
#pragma unroll 1
    for (int r = 0; r < D; r++) {
      Cx<R> acc = {R(0), R(0)};
      const Cx<R>* row = cf + r * D;
#pragma unroll
      for (int c = 0; c < D; c++) acc = cfma(row[c], v[c], acc);
      uint32_t x = b;
#pragma unroll
      for (int i = 0; i < K; i++)
        if ((r >> i) & 1) x |= bit[i];
      s[phys<R>(x)] = acc;
    }
  }
}

template <typename R>
__device__ __forceinline__ void s_diag(Cx<R>* s, int tsz, const DevOp& op, const Cx<R>* cf, uint64_t base,
                                       const Grp& gr) {
  uint32_t xi = 0;
  for (int i = 0; i < op.k; i++)
    if (op.pos[i] == 0xFF) xi |= (uint32_t)((base >> op.gq[i]) & 1ull) << i;
  for (uint32_t a = gr.tid; a < (uint32_t)tsz; a += gr.nthr) {
    if ((a & op.lmask) != op.lval) continue;
    const uint32_t pa = phys<R>(a);
    if (op.kind == OPK_SIGN) {
      s[pa] = Cx<R>{-s[pa].re, -s[pa].im};
    } else {
      uint32_t di = xi;
      for (int i = 0; i < op.k; i++)
        if (op.pos[i] != 0xFF) di |= ((a >> op.pos[i]) & 1u) << i;
      s[pa] = cmul(cf[di], s[pa]);
    }
  }
}

// Anti-diagonal and swap ops of a shared-memory phase (tiles too small for
// register groups).
template <typename R>
__device__ __forceinline__ void s_perm(Cx<R>* s, int tsz, const DevOp& op, const Cx<R>* cf, const Grp& gr) {
  if (op.kind == OPK_ANTIDIAG) {
    const int p = op.pos[0];
    for (uint32_t g = gr.tid; g < (uint32_t)(tsz >> 1); g += gr.nthr) {
      const uint32_t i0 = ins0(g, p);
      if ((i0 & op.lmask) != op.lval) continue;
      const uint32_t a = phys<R>(i0), b = phys<R>(i0 | (1u << p));
      const Cx<R> x = s[a], y = s[b];
      s[a] = cmul(cf[0], y);
      s[b] = cmul(cf[1], x);
    }
  } else {
    for (uint32_t g = gr.tid; g < (uint32_t)(tsz >> 2); g += gr.nthr) {
      const uint32_t b = ins0(ins0(g, op.spos[0]), op.spos[1]);
      if ((b & op.lmask) != op.lval) continue;
      const uint32_t i01 = phys<R>(b | (1u << op.pos[0])), i10 = phys<R>(b | (1u << op.pos[1]));
      const Cx<R> t = s[i01];
      s[i01] = s[i10];
      s[i10] = t;
    }
  }
}

// Global offset of local amplitude l of a tile: local bit i is global bit
// tq[i] (without the tile's base).
__device__ __forceinline__ uint64_t tile_offset(uint32_t l, const ProgramHeader& h) {
  uint64_t off = 0;
#pragma unroll
  for (int i = 0; i < kMaxTileQ; i++) {
    if (i >= h.m) break;
    if ((l >> i) & 1u) off |= 1ull << h.tq[i];
  }
  return off;
}

// Writes the thread's 2^RQ register amplitudes straight to the state: the
// amplitude of register combination j is at g + (XOR of gs[i] over the set
// bits i of j).  With local bit 0 in register slot 0, pairs (j, j+1) are
// adjacent in the state and go out as one 16-byte store (complex64).
template <typename R, int RQ>
__device__ __forceinline__ void reg_store_global(const Cx<R> (&v)[1 << RQ], Cx<R>* __restrict__ state, uint64_t g,
                                                 const uint64_t (&gs)[RQ], bool pairs) {
  if (sizeof(Cx<R>) == 8 && pairs) {
    uint64_t off[(1 << RQ) / 2];
    off[0] = g;
#pragma unroll
    for (int j = 2; j < (1 << RQ); j += 2) {
      const int low = j & -j;
      const int i = low == 2 ? 1 : low == 4 ? 2 : low == 8 ? 3 : 4;
      off[j / 2] = off[(j ^ low) / 2] ^ gs[i];
    }
#pragma unroll
    for (int j = 0; j < (1 << RQ); j += 2)
      *reinterpret_cast<float4*>(state + off[j / 2]) =
          make_float4((float)v[j].re, (float)v[j].im, (float)v[j + 1].re, (float)v[j + 1].im);
  } else {
    uint64_t off[1 << RQ];
    off[0] = g;
#pragma unroll
    for (int j = 1; j < (1 << RQ); j++) {
      const int low = j & -j;
      const int i = low == 1 ? 0 : low == 2 ? 1 : low == 4 ? 2 : low == 8 ? 3 : 4;
      off[j] = off[j ^ low] ^ gs[i];
    }
#pragma unroll
    for (int j = 0; j < (1 << RQ); j++) state[off[j]] = v[j];
  }
}

// Copies a tile from its shared-memory stage (swizzled) to the state, 16
// bytes a thread at a time (the last phase of a direct pass was not a
// register phase).
template <typename R>
__device__ __forceinline__ void stage_copy_out(const Cx<R>* s, int tsz, Cx<R>* __restrict__ gstate, uint64_t base,
                                               const ProgramHeader& h, const Grp& gr) {
  constexpr int A = 16 / sizeof(Cx<R>);
  for (uint32_t v = gr.tid; v < (uint32_t)(tsz / A); v += gr.nthr) {
    const uint32_t l = v * A;
    *reinterpret_cast<uint4*>(gstate + (base | tile_offset(l, h))) = *reinterpret_cast<const uint4*>(s + phys<R>(l));
  }
}

}  // namespace sv
