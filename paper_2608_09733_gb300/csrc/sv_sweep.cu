// sv_sweep.cu -- gate application kernels for sm_103a.
//
// One launch makes one pass over the state (a "sweep").  The state is cut
// into tiles of 2^m amplitudes; a tile is the set of amplitudes whose bits
// outside the tile qubits tq[] are fixed, i.e. the paper's group of amplitudes
// "that differ only on the target qubits" (Sec. 5.3), widened from the k
// targets of one gate to the m qubits of every operation the pass applies.
// Group members are found by bit insertion instead of the paper's index table
// I_T (no 2^n integer array is stored).  The low L tile qubits are 0..L-1, so a
// tile is 2^(m-L) contiguous runs of 2^L amplitudes (256 bytes), read and
// written with coalesced 16-byte accesses.
//
// Inside the tile the ops run in phases.  In a register phase each thread
// holds 16 amplitudes that differ only on four "register" tile qubits and
// applies every consecutive op whose moving qubits are among them with plain
// FMAs on registers: dense and real one-/two-qubit matrices (Sec. 5.3: a real
// gate needs half the products), diagonal gates and sign flips (CZ, Z) which
// move nothing, and X/CNOT/SWAP which only permute registers (Sec. 9.2:
// diagonal and permutation paths).  Shared memory is read and written once per
// phase, with an XOR swizzle of 16-byte granules so the strided register
// groups do not collide in banks.  Dense k >= 3 operations (the paper's fused
// blocks) run group by group straight in shared memory.
#include <cuda_runtime.h>

#include <cstddef>

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
//  - float (issue-bound): three in-place shears a -= t b; b += s a; a -= t b
//    with coef = (t, s) = (tan(alpha/2), sin(alpha)); no temporaries, one
//    packed FMA per shear.
//  - double (FP64-pipe-bound): two FMAs per component in scaled form, the
//    scale carried by a later phase table: coef.re = t and, with COT clear,
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

#define SV_SLOT_CASES(F, FL, ...)                        \
  switch (op.rs[0]) {                                    \
    case 0: F<R, RQ, 0, FL>(__VA_ARGS__); break;         \
    case 1: F<R, RQ, 1, FL>(__VA_ARGS__); break;         \
    case 2: F<R, RQ, 2, FL>(__VA_ARGS__); break;         \
    case 3: F<R, RQ, 3, FL>(__VA_ARGS__); break;         \
    default:                                             \
      if constexpr (RQ > 4) F<R, RQ, 4, FL>(__VA_ARGS__); \
      break;                                             \
  }

#define SV_PAIR_CASES(F, ...)                            \
  switch (op.rs[0] * 8 + op.rs[1]) { /* rs[0] < rs[1] */ \
    case 1: F<R, RQ, 0, 1>(__VA_ARGS__); break;          \
    case 2: F<R, RQ, 0, 2>(__VA_ARGS__); break;          \
    case 3: F<R, RQ, 0, 3>(__VA_ARGS__); break;          \
    case 10: F<R, RQ, 1, 2>(__VA_ARGS__); break;         \
    case 11: F<R, RQ, 1, 3>(__VA_ARGS__); break;         \
    case 19: F<R, RQ, 2, 3>(__VA_ARGS__); break;         \
    case 4: if constexpr (RQ > 4) F<R, RQ, 0, 4>(__VA_ARGS__); break;  \
    case 12: if constexpr (RQ > 4) F<R, RQ, 1, 4>(__VA_ARGS__); break; \
    case 20: if constexpr (RQ > 4) F<R, RQ, 2, 4>(__VA_ARGS__); break; \
    default: if constexpr (RQ > 4) F<R, RQ, 3, 4>(__VA_ARGS__); break; \
  }

#ifndef SV_KRON_FENCE_ON
#define SV_KRON_FENCE_ON 1
#endif
#if SV_KRON_FENCE_ON
#define SV_KRON_FENCE() asm volatile("" ::: "memory")
#else
#define SV_KRON_FENCE() ((void)0)
#endif

// Op sets a pass kernel is compiled for: the code of op kinds a program never
// uses still costs registers and moves, so the launch picks the smallest set.
constexpr int kOpsRot = 0;   // KROT, PHASE (and sign flips)
constexpr int kOpsPerm = 1;  // + anti-diagonal (X, CNOT ...) and SWAP
constexpr int kOpsAll = 2;   // + KRON, dense/real k <= 2, general diagonals

static_assert(offsetof(SweepProgram<float>, coef) % 16 == 0, "16-byte table pairs in a program's pool");

template <typename R, int RQ, int OPS>
__device__ __forceinline__ void apply_reg(Cx<R> (&v)[1 << RQ], const DevOp& op, uint32_t code, const Cx<R>* pool,
                                          uint32_t tb, uint64_t base) {
  const uint32_t fl = (code >> 4) & 7u;
  if ((fl & OPF_XCOND) && (base & op.xmask) != op.xval) return;  // same for the whole block
  if ((fl & OPF_TCOND) && (tb & op.tmask) != op.tval) return;    // same for the thread's amplitudes
  const Cx<R>* cf = pool + (code >> 17);
  const uint32_t rm = (code >> 7) & 31u, rv = (code >> 12) & 31u;
  switch (code & 15u) {
    case OPK_KRON:  // one-qubit gates on distinct slots commute: apply each present block
      // (the fences keep one block's coefficients live at a time)
      if constexpr (OPS >= kOpsAll) {
      if (rm & 1u) r_u1<R, RQ, 0>(v, cf);
      SV_KRON_FENCE();
      if (rm & 2u) r_u1<R, RQ, 1>(v, cf + 4);
      SV_KRON_FENCE();
      if (rm & 4u) r_u1<R, RQ, 2>(v, cf + 8);
      SV_KRON_FENCE();
      if (rm & 8u) r_u1<R, RQ, 3>(v, cf + 12);
      if constexpr (RQ > 4) {
        SV_KRON_FENCE();
        if (rm & 16u) r_u1<R, RQ, 4>(v, cf + 16);
      }
      }
      break;
    case OPK_KROT:  // rotations on distinct slots commute
      if (rm & 1u) r_rot_slot<R, RQ, 0>(v, cf, rv);
      SV_KRON_FENCE();
      if (rm & 2u) r_rot_slot<R, RQ, 1>(v, cf, rv);
      SV_KRON_FENCE();
      if (rm & 4u) r_rot_slot<R, RQ, 2>(v, cf, rv);
      SV_KRON_FENCE();
      if (rm & 8u) r_rot_slot<R, RQ, 3>(v, cf, rv);
      if constexpr (RQ > 4) {
        SV_KRON_FENCE();
        if (rm & 16u) r_rot_slot<R, RQ, 4>(v, cf, rv);
      }
      break;
    case OPK_PHASE: {
      // variant of the table picked by the selector bits (thread bits, or
      // bits outside the tile); variants are table_stride entries apart
      uint32_t var = 0;
      for (int i = 0; i < op.k; i++) {
        const uint32_t c = op.gq[i];
        const uint32_t b = c < 64 ? (tb >> c) & 1u : (uint32_t)(base >> (c - 64)) & 1u;
        var |= b << i;
      }
      const Cx<R>* T0 = cf + var * (uint32_t)table_stride<R>(RQ);
      // v *= T with one temporary: everything else in place
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
      break;
    }
    case OPK_DENSE:
    case OPK_REAL:
      if constexpr (OPS >= kOpsAll) {
      if (op.k == 1) {
        if ((code & 15u) == OPK_REAL) {
          SV_SLOT_CASES(r_dense1, true, v, cf, rm, rv)
        } else {
          SV_SLOT_CASES(r_dense1, false, v, cf, rm, rv)
        }
      } else {
        SV_PAIR_CASES(r_dense2, v, cf, rm, rv)
      }
      }
      break;
    case OPK_ANTIDIAG:
      if constexpr (OPS >= kOpsPerm) {
      if (fl & OPF_FLIP) {  // pure bit flip (X, CNOT): no multiplies
        SV_SLOT_CASES(r_anti1, true, v, cf, rm, rv)
      } else {
        SV_SLOT_CASES(r_anti1, false, v, cf, rm, rv)
      }
      }
      break;
    case OPK_SWAP:
      if constexpr (OPS >= kOpsPerm) { SV_PAIR_CASES(r_swap, v, rm, rv) }
      break;
    case OPK_DIAG:
      if constexpr (OPS >= kOpsAll) r_diag<R, RQ>(v, op, cf, tb, base);
      break;
    default: break;
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

template <typename R, int K>
__device__ __forceinline__ void s_denseK(Cx<R>* s, int tsz, const DevOp& op, const Cx<R>* cf) {
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
__device__ __forceinline__ void s_diag(Cx<R>* s, int tsz, const DevOp& op, const Cx<R>* cf, uint64_t base) {
  uint32_t xi = 0;
  for (int i = 0; i < op.k; i++)
    if (op.pos[i] == 0xFF) xi |= (uint32_t)((base >> op.gq[i]) & 1ull) << i;
  for (uint32_t a = threadIdx.x; a < (uint32_t)tsz; a += blockDim.x) {
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
__device__ __forceinline__ void s_perm(Cx<R>* s, int tsz, const DevOp& op, const Cx<R>* cf) {
  if (op.kind == OPK_ANTIDIAG) {
    const int p = op.pos[0];
    for (uint32_t g = threadIdx.x; g < (uint32_t)(tsz >> 1); g += blockDim.x) {
      const uint32_t i0 = ins0(g, p);
      if ((i0 & op.lmask) != op.lval) continue;
      const uint32_t a = phys<R>(i0), b = phys<R>(i0 | (1u << p));
      const Cx<R> x = s[a], y = s[b];
      s[a] = cmul(cf[0], y);
      s[b] = cmul(cf[1], x);
    }
  } else {
    for (uint32_t g = threadIdx.x; g < (uint32_t)(tsz >> 2); g += blockDim.x) {
      const uint32_t b = ins0(ins0(g, op.spos[0]), op.spos[1]);
      if ((b & op.lmask) != op.lval) continue;
      const uint32_t i01 = phys<R>(b | (1u << op.pos[0])), i10 = phys<R>(b | (1u << op.pos[1]));
      const Cx<R> t = s[i01];
      s[i01] = s[i10];
      s[i10] = t;
    }
  }
}

// ---------------------------------------------------------------- kernels

// Runs every phase of a program on a tile that is already in shared memory.
// KMAX: widest dense operation the program runs in shared memory; RQ: the
// register qubits of its register phases.
template <typename R, int KMAX, int RQ, int OPS>
__device__ __forceinline__ void run_phases(const SweepProgram<R>& P, const Cx<R>* coef, Cx<R>* s, int tsz,
                                           uint64_t base) {
  const ProgramHeader& h = P.h;
  for (int p = 0; p < h.nphases; p++) {
    const Phase& ph = P.ph[p];
    if (ph.kind == PH_REG) {
      if (threadIdx.x < (1u << ph.ntpos)) {
        // thread bits: the thread index with zeros inserted at the register
        // positions (rp[] ascending), i.e. deposited into tpos[]
        uint32_t tb = threadIdx.x;
        uint32_t m[RQ];
#pragma unroll
        for (int i = 0; i < RQ; i++) {
          m[i] = 1u << ph.rp[i];
          tb = ins0(tb, ph.rp[i]);
        }
        Cx<R> v[1 << RQ];
        reg_load<R, RQ>(v, s, tb, m);
        // Sign flips commute with each other: a run of them becomes one mask of
        // the thread's amplitudes to negate, applied before the next other op.
        uint32_t neg = 0;
        // each op's dispatch word is loaded one op ahead, off the critical path
        const DevOp* ops = P.ops + ph.first;
        const int nops = ph.nops;
        uint32_t code_next = nops ? ops[0].pad : 0u;
        for (int i = 0; i < nops; i++) {
          const uint32_t code = code_next;
          if (i + 1 < nops) code_next = ops[i + 1].pad;
          const DevOp& op = ops[i];
          if ((code & 15u) == OPK_SIGN) {  // op.coef holds the precomputed pattern
            bool on = true;
            if (code & (OPF_XCOND << 4)) on = (base & op.xmask) == op.xval;
            if (code & (OPF_TCOND << 4)) on = on && (tb & op.tmask) == op.tval;
            if (on) neg ^= op.coef;
            continue;
          }
          if (neg) {
            apply_neg<R, RQ>(v, neg);
            neg = 0;
          }
          apply_reg<R, RQ, OPS>(v, op, code, coef, tb, base);
        }
        if (neg) apply_neg<R, RQ>(v, neg);
        reg_store<R, RQ>(v, s, tb, m);
      }
    } else {
      const DevOp& op = P.ops[ph.first];
      if ((base & op.xmask) == op.xval) {
        const Cx<R>* cf = coef + op.coef;
        switch (op.kind) {
          case OPK_DIAG:
          case OPK_SIGN: s_diag<R>(s, tsz, op, cf, base); break;
          case OPK_ANTIDIAG:
          case OPK_SWAP: s_perm<R>(s, tsz, op, cf); break;
          default:
            switch (op.k) {
              case 1: s_denseK<R, 1>(s, tsz, op, cf); break;
              case 2: s_denseK<R, 2>(s, tsz, op, cf); break;
              case 3: if constexpr (KMAX >= 3) s_denseK<R, 3>(s, tsz, op, cf); break;
              case 4: if constexpr (KMAX >= 4) s_denseK<R, 4>(s, tsz, op, cf); break;
              default: if constexpr (KMAX >= 5) s_denseK<R, 5>(s, tsz, op, cf); break;
            }
        }
      }
    }
    __syncthreads();
  }
}

// Asynchronous 16-byte global -> shared copy (completes at cp_async_wait).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

#ifndef SV_SWEEP_MIN_BLOCKS
#define SV_SWEEP_MIN_BLOCKS 3  // complex64, four register qubits: resident CTAs per SM
#endif
// Launch shape of the five-register-qubit (32 amplitudes per thread) passes:
// largest block, resident CTAs per SM hint, and whether tiles are double-buffered.
// The bound of 256 threads x 2 CTAs caps the kernel at 128 registers, which
// also lets four 128-thread CTAs (12-qubit complex64 tiles, 32 KiB each) share
// an SM: a CTA waiting at a barrier or for its tile's copies then leaves three
// others to issue.
#ifndef SV_RQ5_MAXT
#define SV_RQ5_MAXT 256
#endif
#ifndef SV_RQ5_MINB
#define SV_RQ5_MINB 2
#endif
#ifndef SV_RQ5_DBUF
#define SV_RQ5_DBUF false
#endif

// One pass over the state.  With DBUF each CTA walks its tiles with two
// shared-memory buffers: while it runs the program on tile t, the copies of
// tile t + grid are already in flight (cp.async), so the gather latency hides
// behind the arithmetic.  Without DBUF (tiles too large for two buffers) the
// copies of a tile are waited for before it runs.  Each tile is scattered back
// with 16-byte stores.
template <typename R, int KMAX, int RQ, bool DBUF, int OPS>
__global__ void __launch_bounds__(RQ == 5 ? SV_RQ5_MAXT : 256,
                                  sizeof(R) == 4 ? (RQ == 5 ? SV_RQ5_MINB : SV_SWEEP_MIN_BLOCKS) : 1)
    k_sweep(Cx<R>* __restrict__ state, const __grid_constant__ SweepProgram<R> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ProgramHeader& h = P.h;
  const int tsz = 1 << h.m;
  Cx<R>* buf[2] = {reinterpret_cast<Cx<R>*>(smem_raw), reinterpret_cast<Cx<R>*>(smem_raw) + (DBUF ? tsz : 0)};
  constexpr int A = 16 / sizeof(Cx<R>);  // amplitudes per 16-byte access
  const int nvec = tsz / A;
  const uint64_t ntiles = 1ull << (h.n - h.m);
  // global offset of every run of 2^L contiguous amplitudes of a tile (the
  // same for all tiles), kept after the buffers
  uint64_t* hi_off = reinterpret_cast<uint64_t*>(buf[1] + tsz);
  const int nhi = 1 << (h.m - h.L);
  for (int c = threadIdx.x; c < nhi; c += blockDim.x) hi_off[c] = local_offset((uint32_t)c << h.L, h);
  // the coefficient pool, staged once per CTA (broadcast reads from shared
  // memory), 16-byte aligned
  Cx<R>* scoef = reinterpret_cast<Cx<R>*>(hi_off + nhi + (nhi & 1));
  for (int c = threadIdx.x; c < h.ncoef; c += blockDim.x) scoef[c] = P.coef[c];
  const uint32_t lowmask = (1u << h.L) - 1u;
  __syncthreads();
  auto tile_base = [&](uint64_t tile) {
    uint64_t base = tile;
    for (int i = 0; i < h.m; i++) base = ins0_64(base, h.tq[i]);
    return base;
  };
  auto gather = [&](Cx<R>* s, uint64_t base) {
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
      const uint32_t l = (uint32_t)(v * A);
      cp_async16(s + phys<R>(l), state + (base + (hi_off[l >> h.L] | (l & lowmask))));
    }
    cp_async_commit();
  };
  uint64_t tile = blockIdx.x;
  if (DBUF && tile < ntiles) gather(buf[0], tile_base(tile));
  for (int cur = 0; tile < ntiles; tile += gridDim.x, cur ^= (DBUF ? 1 : 0)) {
    const uint64_t base = tile_base(tile);
    if constexpr (DBUF) {
      const uint64_t next = tile + gridDim.x;
      if (next < ntiles) {
        gather(buf[cur ^ 1], tile_base(next));
        cp_async_wait<1>();  // this thread's copies of the current tile are done
      } else {
        cp_async_wait<0>();
      }
    } else {
      gather(buf[0], base);
      cp_async_wait<0>();
    }
    __syncthreads();  // ... and every thread's
    Cx<R>* s = buf[cur];
    run_phases<R, KMAX, RQ, OPS>(P, scoef, s, tsz, base);
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
      const uint32_t l = (uint32_t)(v * A);
      *reinterpret_cast<uint4*>(state + (base + (hi_off[l >> h.L] | (l & lowmask)))) =
          *reinterpret_cast<const uint4*>(s + phys<R>(l));
    }
    __syncthreads();  // the buffer is free for the next copies
  }
}

// Packed small states (serving): CTA b simulates request b entirely in shared
// memory -- |0..0>, every program of the request, then sum_q <Z_q> =
// sum_a |psi_a|^2 (n - 2 popcount(a)) -- and writes one double.  The state
// never touches HBM.
template <typename R>
__global__ void __launch_bounds__(256) k_small_batch(const SweepProgram<R>* __restrict__ progs,
                                                     const int* __restrict__ first_prog, const int* __restrict__ nq,
                                                     double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<R>* s = reinterpret_cast<Cx<R>*>(smem_raw);
  __shared__ double red[8];
  const int b = blockIdx.x;
  const int n = nq[b];
  const int tsz = 1 << n;
  for (int a = threadIdx.x; a < tsz; a += blockDim.x) s[phys<R>(a)] = Cx<R>{R(a == 0 ? 1 : 0), R(0)};
  __syncthreads();
  for (int p = first_prog[b]; p < first_prog[b + 1]; p++)
    run_phases<R, 5, kRegQ, kOpsAll>(progs[p], progs[p].coef, s, tsz, 0ull);
  double acc = 0.0;
  for (int a = threadIdx.x; a < tsz; a += blockDim.x) {
    const Cx<R> x = s[phys<R>(a)];
    acc += (double)(x.re * x.re + x.im * x.im) * (double)(n - 2 * __popc(a));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
    out[b] = t;
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

int sweep_threads(int m, int rq) {
  // one thread per register group of 2^rq amplitudes; at least one warp
  return m - rq >= 5 ? (1 << (m - rq)) : 32;
}

template <typename R, int KMAX, int RQ, bool DBUF, int OPS>
static cudaError_t launch_sweep_k(Cx<R>* state, const SweepProgram<R>& prog, cudaStream_t stream) {
  const int smem = ((int)sizeof(Cx<R>) << (prog.h.m + (DBUF ? 1 : 0))) + (8 << (prog.h.m - prog.h.L)) + 8 +
                   (int)sizeof(Cx<R>) * prog.h.ncoef;
  // raise the dynamic shared-memory limit to what this launch needs (per device)
  static int configured_bytes[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem > 48 * 1024 && smem > configured_bytes[dev]) {
    cudaError_t e =
        cudaFuncSetAttribute(k_sweep<R, KMAX, RQ, DBUF, OPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured_bytes[dev] = smem;
  }
  const int threads = sweep_threads(prog.h.m, RQ);
  if (threads > (RQ == 5 ? SV_RQ5_MAXT : 256)) return cudaErrorInvalidConfiguration;  // a group per thread
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<R, KMAX, RQ, DBUF, OPS>, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t ntiles = 1ull << (prog.h.n - prog.h.m);
  uint64_t grid = (uint64_t)device_sm_count() * per_sm;
  if (grid > ntiles) grid = ntiles;
  k_sweep<R, KMAX, RQ, DBUF, OPS><<<(unsigned)grid, threads, smem, stream>>>(state, prog);
  return cudaGetLastError();
}

template <typename R, int RQ, bool DBUF>
static cudaError_t launch_sweep_rq(Cx<R>* state, const SweepProgram<R>& prog, cudaStream_t stream) {
  int kmax = 1;
  bool perm = false, other = false;
  for (int p = 0; p < prog.h.nphases; p++) {
    const Phase& ph = prog.ph[p];
    if (ph.kind != PH_SMEM) {
      for (int o = ph.first; o < ph.first + ph.nops; o++) {
        const uint32_t kind = prog.ops[o].pad & 15u;
        if (kind == OPK_ANTIDIAG || kind == OPK_SWAP)
          perm = true;
        else if (kind != OPK_KROT && kind != OPK_PHASE && kind != OPK_SIGN)
          other = true;
      }
      continue;
    }
    const DevOp& op = prog.ops[ph.first];
    if ((op.kind == OPK_DENSE || op.kind == OPK_REAL) && op.k > kmax) kmax = op.k;
  }
  if (kmax <= 2 && !other) {
    if (!perm) return launch_sweep_k<R, 2, RQ, DBUF, kOpsRot>(state, prog, stream);
    return launch_sweep_k<R, 2, RQ, DBUF, kOpsPerm>(state, prog, stream);
  }
  if (kmax <= 2) return launch_sweep_k<R, 2, RQ, DBUF, kOpsAll>(state, prog, stream);
  if (kmax == 3) return launch_sweep_k<R, 3, RQ, DBUF, kOpsAll>(state, prog, stream);
  return launch_sweep_k<R, 5, RQ, DBUF, kOpsAll>(state, prog, stream);
}

template <typename R>
cudaError_t launch_sweep(Cx<R>* state, const SweepProgram<R>& prog, cudaStream_t stream) {
  // four register qubits with two tile buffers, or five with one (12-qubit
  // complex64 tiles; complex128 tiles have 11 qubits)
  if constexpr (sizeof(R) == 4)
    if (prog.h.rq == 5) return launch_sweep_rq<R, 5, SV_RQ5_DBUF>(state, prog, stream);
  if (prog.h.rq != 4) return cudaErrorInvalidValue;
  return launch_sweep_rq<R, 4, true>(state, prog, stream);
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

template <typename R>
cudaError_t launch_small_batch(const SweepProgram<R>* progs, const int* first_prog, const int* nq, int n_requests,
                               int max_n, double* out, cudaStream_t stream) {
  const int smem = (int)sizeof(Cx<R>) << max_n;
  static int configured_bytes[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem > 48 * 1024 && smem > configured_bytes[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_small_batch<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured_bytes[dev] = smem;
  }
  k_small_batch<R><<<n_requests, 256, smem, stream>>>(progs, first_prog, nq, out);
  return cudaGetLastError();
}

template cudaError_t launch_small_batch<float>(const SweepProgram<float>*, const int*, const int*, int, int, double*,
                                               cudaStream_t);
template cudaError_t launch_small_batch<double>(const SweepProgram<double>*, const int*, const int*, int, int, double*,
                                                cudaStream_t);
template cudaError_t launch_sweep<float>(Cx<float>*, const SweepProgram<float>&, cudaStream_t);
template cudaError_t launch_sweep<double>(Cx<double>*, const SweepProgram<double>&, cudaStream_t);
template cudaError_t launch_init_basis<float>(Cx<float>*, int, uint64_t, cudaStream_t);
template cudaError_t launch_init_basis<double>(Cx<double>*, int, uint64_t, cudaStream_t);

}  // namespace sv
