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
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdlib>
#include <mutex>

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

// ---------------------------------------------------------------- kernels

// Runs every phase of a program on a tile that is already in shared memory.
// KMAX: widest dense operation the program runs in shared memory; RQ: the
// register qubits of its register phases.
struct NoRelease {
  __device__ __forceinline__ void operator()() const {}
};

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

// Runs every phase of a program on a tile that is already in shared memory.
// KMAX: widest dense operation the program runs in shared memory; RQ: the
// register qubits of its register phases.
//
// DIRECT (TMA pass): the tile goes back to the state from the last phase
// instead of staying in shared memory.  A last register phase loads its
// registers, meets the group's barrier, calls release() (the stage is free:
// the caller refills it) and writes its results straight to `gstate` at the
// tile's `base`; any other last phase is followed by a copy of the stage to
// the state, a barrier and release().
template <typename R, int KMAX, int RQ, int OPS, bool DIRECT = false, typename Release = NoRelease>
__device__ __forceinline__ void run_phases(const SweepProgram<R>& P, const Cx<R>* coef, Cx<R>* s, int tsz,
                                           uint64_t base, const Grp& gr, Cx<R>* gstate = nullptr,
                                           const Release& release = Release()) {
  const ProgramHeader& h = P.h;
  for (int p = 0; p < h.nphases; p++) {
    const Phase& ph = P.ph[p];
    const bool direct = DIRECT && p == h.nphases - 1 && ph.kind == PH_REG;
    if (ph.kind == PH_REG) {
      const bool active = gr.tid < (1u << ph.ntpos);
      // thread bits: the thread index with zeros inserted at the register
      // positions (rp[] ascending), i.e. deposited into tpos[]
      uint32_t tb = gr.tid;
      uint32_t m[RQ];
#pragma unroll
      for (int i = 0; i < RQ; i++) {
        m[i] = 1u << ph.rp[i];
        tb = ins0(tb, ph.rp[i]);
      }
      Cx<R> v[1 << RQ];
      if (active) reg_load<R, RQ>(v, s, tb, m);
      if (direct) {
        grp_sync(gr);  // every thread has its registers: the stage is free
        release();
      }
      if (active) {
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
        if (direct) {
          uint64_t gs[RQ];
#pragma unroll
          for (int i = 0; i < RQ; i++) gs[i] = 1ull << h.tq[ph.rp[i]];
          reg_store_global<R, RQ>(v, gstate, base | tile_offset(tb, h), gs, m[0] == 1u);
        } else {
          reg_store<R, RQ>(v, s, tb, m);
        }
      }
      if (direct) return;
    } else {
      const DevOp& op = P.ops[ph.first];
      if ((base & op.xmask) == op.xval) {
        const Cx<R>* cf = coef + op.coef;
        switch (op.kind) {
          case OPK_DIAG:
          case OPK_SIGN: s_diag<R>(s, tsz, op, cf, base, gr); break;
          case OPK_ANTIDIAG:
          case OPK_SWAP: s_perm<R>(s, tsz, op, cf, gr); break;
          default:
            switch (op.k) {
              case 1: s_denseK<R, 1>(s, tsz, op, cf, gr); break;
              case 2: s_denseK<R, 2>(s, tsz, op, cf, gr); break;
              case 3: if constexpr (KMAX >= 3) s_denseK<R, 3>(s, tsz, op, cf, gr); break;
              case 4: if constexpr (KMAX >= 4) s_denseK<R, 4>(s, tsz, op, cf, gr); break;
              default: if constexpr (KMAX >= 5) s_denseK<R, 5>(s, tsz, op, cf, gr); break;
            }
        }
      }
    }
    grp_sync(gr);
  }
  if constexpr (DIRECT) {  // the last phase was not a register phase: copy the stage out
    constexpr int A = 16 / sizeof(Cx<R>);
    for (uint32_t v = gr.tid; v < (uint32_t)(tsz / A); v += gr.nthr) {
      const uint32_t l = v * A;
      *reinterpret_cast<uint4*>(gstate + (base | tile_offset(l, h))) = *reinterpret_cast<const uint4*>(s + phys<R>(l));
    }
    grp_sync(gr);
    release();
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
    run_phases<R, KMAX, RQ, OPS>(P, scoef, s, tsz, base, Grp{threadIdx.x, blockDim.x, 0u});
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
      const uint32_t l = (uint32_t)(v * A);
      *reinterpret_cast<uint4*>(state + (base + (hi_off[l >> h.L] | (l & lowmask)))) =
          *reinterpret_cast<const uint4*>(s + phys<R>(l));
    }
    __syncthreads();  // the buffer is free for the next copies
  }
}

// ---------------------------------------------------------------- TMA pass
//
// The same pass as k_sweep with the tile movement done by the tensor memory
// accelerator.  One CTA per SM walks its tiles (tile = blockIdx.x + k *
// gridDim.x) through a ring of `ns` shared-memory stages (tile k in stage
// k mod ns):
//   - a tile is 16 boxes of 2 KiB, each box the 2^(E+4) amplitudes of local
//     bits 0..E+3, where 2^E amplitudes make one 128-byte row (E = 4 for
//     complex64, 3 for complex128).  A five-dimensional tensor map per pass
//     describes the state as [2^(n-q3)][2^(q3-q2)][2^(q2-q1)][2^(q1-E)][row],
//     q1..q3 being the tile qubits at local positions E+1..E+3; a box takes
//     two entries of each outer dimension.  The 128-byte swizzle of the copies
//     places amplitude l at phys(l), the XOR layout the register phases read;
//   - NC groups of 2^(m-RQ) threads each take every NC-th tile: wait for its
//     stage to fill, run the program's phases on it (a named barrier per
//     group), then thread 0 of the group stores the stage back with TMA, waits
//     until the store has read shared memory, and refills the stage with the
//     tile ns places further on.
// So ns - NC tiles are loading while the groups compute, and no compute
// thread spends instructions on addresses or 16-byte copies.  There is no
// separate producer warp: a 17th warp would cap the compute threads' registers
// at 96 (the register file is split between the SM's four schedulers).
//
// Every wait is bounded (one second of %globaltimer): a wait that runs out
// records SV_ERR_TIMEOUT in g_sweep_status, the CTA's groups stop, and the
// copies already issued are waited for (bounded) before the CTA exits.

__device__ int g_sweep_status = 0;  // SV_OK, or the first error a pass kernel recorded

constexpr uint64_t kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of parity `parity` to complete, for at most
// kWaitLimitNs.  Gives up early when another thread of the CTA has already
// given up (*cta_flag != 0; pass NULL to wait regardless).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, volatile int* cta_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; it++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 15u) == 0) {
      if (cta_flag && *cta_flag) return false;
      if (global_ns() - t0 > kWaitLimitNs) {
        atomicCAS(&g_sweep_status, 0, (int)SV_ERR_TIMEOUT);
        if (cta_flag) *cta_flag = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const volatile uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];\n" : "=r"(v) : "r"(smem_u32((const void*)p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(volatile uint32_t* p, uint32_t v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;\n" ::"r"(smem_u32((const void*)p)), "r"(v) : "memory");
}
// Waits until *tag == want (read with acquire), for at most kWaitLimitNs
// (give-up rules as mbar_wait_bounded).
__device__ __forceinline__ bool tag_wait_bounded(const volatile uint32_t* tag, uint32_t want, volatile int* cta_flag) {
  if (ld_acquire_u32(tag) == want) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; it++) {
    if (ld_acquire_u32(tag) == want) return true;
    if ((it & 15u) == 0) {
      if (*cta_flag) return false;
      if (global_ns() - t0 > kWaitLimitNs) {
        atomicCAS(&g_sweep_status, 0, (int)SV_ERR_TIMEOUT);
        *cta_flag = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void tma_load5(uint32_t dst, const void* map, int c1, int c2, int c3, int c4,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}
// Box geometry of a pass, passed beside its tensor map: the tile qubits at
// local positions E+1..E+3 (q1..q3) and above E+3 (hq[], the box index bits).
struct TmaBoxes {
  int q1, q2, q3;
  int nhq;
  int hq[kMaxTileQ];
};

template <typename R>
__device__ __forceinline__ void tma_coords(uint64_t g, const TmaBoxes& bx, int& c1, int& c2, int& c3, int& c4) {
  constexpr int E = sizeof(Cx<R>) == 8 ? 4 : 3;
  c1 = (int)((g >> E) & ((1ull << (bx.q1 - E)) - 1ull));
  c2 = (int)((g >> bx.q1) & ((1ull << (bx.q2 - bx.q1)) - 1ull));
  c3 = (int)((g >> bx.q2) & ((1ull << (bx.q3 - bx.q2)) - 1ull));
  c4 = (int)(g >> bx.q3);
}

constexpr int kTmaBoxBytes = 2048;
// Threads of a group: 2^(m - RQ), 128 for 12-qubit tiles with five register
// qubits (32 amplitudes a thread).  Sixteen amplitudes a thread (256-thread
// groups, 24 warps an SM at 80 registers) measured slower: 7.55 against 5.65
// ms per 30-qubit pass, the per-phase work of a thread spread over half the
// amplitudes and a third more phases.
template <int RQ>
constexpr int tma_group_threads() {
  return RQ == 5 ? 128 : 256;
}
constexpr int kTmaMaxStages = 8;
static_assert(kTmaMaxStages * 8 % 16 == 0 && 2 * kTmaMaxStages + 1 <= 20, "TMA pass shared-memory layout");

template <typename R, int KMAX, int RQ, int OPS, int NC>
__global__ void __launch_bounds__(NC * tma_group_threads<RQ>(), 1)
    k_sweep_tma(Cx<R>* __restrict__ state, const __grid_constant__ CUtensorMap tmap,
                const __grid_constant__ TmaBoxes bx, const __grid_constant__ SweepProgram<R> P, int ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ProgramHeader& h = P.h;
  constexpr uint32_t T = tma_group_threads<RQ>();
  const int tsz = 1 << h.m;
  const uint32_t tile_bytes = (uint32_t)sizeof(Cx<R>) << h.m;
  // stages from the first 1024-byte boundary (the swizzle pattern's period),
  // then the coefficient pool, the stage barriers, the loads issued into each
  // stage and the CTA's give-up flag
  const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
  unsigned char* stages = smem_raw + pad;
  Cx<R>* scoef = reinterpret_cast<Cx<R>*>(stages + (size_t)ns * tile_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(scoef + ((h.ncoef + 1) & ~1));
  unsigned* issued = reinterpret_cast<unsigned*>(bars + kTmaMaxStages);
  volatile uint32_t* stage_tile = reinterpret_cast<volatile uint32_t*>(issued + kTmaMaxStages);
  volatile int* flag = reinterpret_cast<volatile int*>(stage_tile + kTmaMaxStages);
  // per-CTA constants kept in shared memory rather than in every thread's
  // registers: the deposit mask and steps, and the coordinate offsets of each
  // box of a tile
  // (bars is 16-byte aligned: the pool before it holds an even number of
  // 8-byte complex64 entries or 16-byte complex128 ones; issued is 64 bytes
  // further, cst 80 bytes after issued and boxc 32 after cst, all 16-aligned)
  uint64_t* cst = reinterpret_cast<uint64_t*>(issued + 20);
  int4* boxc = reinterpret_cast<int4*>(cst + 4);
  const uint32_t full0 = smem_u32(bars), st0 = smem_u32(stages);
  const uint64_t ntiles = 1ull << (h.n - h.m);
  const uint64_t K = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  // The base of tile t is t with zeros inserted at the tile qubits (its bits
  // deposited into the other positions, mask M).  Deposits add without
  // unpacking: dep(t + d) = ((dep(t) | ~M) + dep(d)) & M, the carries running
  // through the tile positions set to one.
  auto deposit = [&](uint64_t t) {
    for (int i = 0; i < h.m; i++) t = ins0_64(t, h.tq[i]);
    return t;
  };
  auto dep_add = [&](uint64_t a, uint64_t d) {
    const uint64_t M = cst[0];
    return ((a | ~M) + d) & M;
  };
  auto tile_base = [&](uint64_t k) { return deposit(blockIdx.x + k * gridDim.x); };
  // Lane j < 2^nhq of a loading warp copies box j of a tile: its coordinates
  // are those of the tile's base plus those of the box's own bits (the bit
  // fields are disjoint, so the sum has no carries).
  const uint32_t lane = threadIdx.x & 31u;
  const int nbox = 1 << bx.nhq;
  // One warp fills stage b with tile k (base `base`).  The stage's tag names
  // the tile its barrier's current phase belongs to: groups take tiles
  // round-robin, so a group can reach tile k + 2 ns while the load of tile
  // k + ns into the same stage is still to come, and the barrier's phase
  // parity alone would not tell those two apart.
  auto load_tile = [&](uint32_t b, uint64_t k, uint64_t base) {
    if (lane == 0) {
      issued[b] += 1;
      st_release_u32(stage_tile + b, (uint32_t)k);
      mbar_expect_tx(full0 + 8 * b, tile_bytes);
    }
    __syncwarp();
    if ((int)lane < nbox) {
      int c1, c2, c3, c4;
      tma_coords<R>(base, bx, c1, c2, c3, c4);
      const int4 bc = boxc[lane];
      tma_load5(st0 + b * tile_bytes + lane * kTmaBoxBytes, &tmap, c1 + bc.x, c2 + bc.y, c3 + bc.z, c4 + bc.w,
                full0 + 8 * b);
    }
  };
  for (int c = threadIdx.x; c < h.ncoef; c += blockDim.x) scoef[c] = P.coef[c];
  if (threadIdx.x == 0) {
    *flag = 0;
    for (int b = 0; b < ns; b++) {
      mbar_init(full0 + 8 * b, 1);
      issued[b] = 0;
      stage_tile[b] = 0xFFFFFFFFu;
    }
    cst[0] = deposit((1ull << (h.n - h.m)) - 1ull);
    cst[1] = deposit((uint64_t)NC * gridDim.x);
    cst[2] = deposit((uint64_t)ns * gridDim.x);
    fence_mbar_init();
  }
  if (threadIdx.x < 32 && (int)threadIdx.x < nbox) {
    uint64_t gb = 0;
    for (int i = 0; i < bx.nhq; i++) gb |= (uint64_t)((threadIdx.x >> i) & 1u) << bx.hq[i];
    int4 bc;
    tma_coords<R>(gb, bx, bc.x, bc.y, bc.z, bc.w);
    boxc[threadIdx.x] = bc;
  }
  __syncthreads();
  if (threadIdx.x < 32)  // first fill of the ring
    for (uint64_t k = 0; k < K && k < (uint64_t)ns; k++) load_tile((uint32_t)k, k, tile_base(k));
  const uint32_t g = threadIdx.x / T;
  const Grp gr{threadIdx.x % T, T, 1u + g};
  const bool loader = gr.tid < 32;  // warp 0 of the group refills the stages it frees
  uint64_t base = tile_base(g);
  for (uint64_t k = g; k < K; k += NC, base = dep_add(base, cst[1])) {
    const uint32_t b = (uint32_t)(k % (uint64_t)ns);
    // a wait that runs out sets the CTA's flag and the group carries on over
    // whatever the stage holds: every thread keeps meeting the group's
    // barriers, so nothing waits forever, and the status says the pass failed
    if (tag_wait_bounded(stage_tile + b, (uint32_t)k, flag))
      mbar_wait_bounded(full0 + 8 * b, (uint32_t)((k / ns) & 1), flag);
    auto release = [&]() {
      if (loader && k + ns < K && __all_sync(0xffffffffu, *flag == 0)) load_tile(b, k + ns, dep_add(base, cst[2]));
    };
    run_phases<R, KMAX, RQ, OPS, true>(P, scoef, reinterpret_cast<Cx<R>*>(stages + (size_t)b * tile_bytes), tsz,
                                       base, gr, state, release);
  }
  __syncthreads();
  if (threadIdx.x == 0 && *flag)  // stopped early: loads still in flight must land first
    for (int b = 0; b < ns; b++)
      if (issued[b]) mbar_wait_bounded(full0 + 8 * b, (issued[b] - 1) & 1u, nullptr);
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
    run_phases<R, 5, kRegQ, kOpsAll>(progs[p], progs[p].coef, s, tsz, 0ull, Grp{threadIdx.x, blockDim.x, 0u});
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

// Persistent packed small states (serving): a session kernel whose CTAs take
// requests from a work queue the host fills while it runs.  The queue, its
// published count and the exit flag live in pinned host memory mapped into the
// device; the programs in device memory.  CTA loop: claim the next ticket
// (atomicAdd on the device-side head), wait until the host has published it
// or asked the session to end, run the request's programs on its state in
// shared memory from |0..0>, write sum_q <Z_q> and then the ticket's done word
// (system-scope fence between them).  The wait is bounded by `limit_ns` of
// %globaltimer: when it runs out the CTA records SV_ERR_TIMEOUT in *status
// and returns (an idle session ends this way too).
template <typename R>
__device__ __forceinline__ void run_small_request(const SweepProgram<R>* progs, int first, int last, int n,
                                                  Cx<R>* s, double* red, double& result) {
  const int tsz = 1 << n;
  for (int a = threadIdx.x; a < tsz; a += blockDim.x) s[phys<R>(a)] = Cx<R>{R(a == 0 ? 1 : 0), R(0)};
  __syncthreads();
  const Grp gr{threadIdx.x, blockDim.x, 0u};
  for (int p = first; p < last; p++) {
    if (progs[p].h.rq == 5) {
      if constexpr (sizeof(R) == 4) run_phases<R, 5, 5, kOpsAll>(progs[p], progs[p].coef, s, tsz, 0ull, gr);
    } else {
      run_phases<R, 5, kRegQ, kOpsAll>(progs[p], progs[p].coef, s, tsz, 0ull, gr);
    }
  }
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
    result = t;
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_small_session(SmallSessionDev d, const SweepProgram<R>* __restrict__ progs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<R>* s = reinterpret_cast<Cx<R>*>(smem_raw);
  __shared__ double red[8];
  __shared__ long long s_ticket;
  __shared__ int s_stop;
  __shared__ double s_result;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long t = (long long)atomicAdd(d.head, 1ull);
      int stop = 0;
      const uint64_t t0 = global_ns();
      for (uint32_t it = 0;; it++) {
        long long pub;
        asm volatile("ld.acquire.sys.global.s64 %0, [%1];" : "=l"(pub) : "l"(d.tail) : "memory");
        if (t < pub) break;
        int ex;
        asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(ex) : "l"(d.exit_flag) : "memory");
        if (ex) {
          stop = 1;
          break;
        }
        if ((it & 15u) == 15u && global_ns() - t0 > d.limit_ns) {
          atomicCAS(d.status, 0, (int)SV_ERR_TIMEOUT);
          stop = 1;
          break;
        }
        __nanosleep(2000);
      }
      s_ticket = t;
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) return;
    const long long t = s_ticket;
    const SmallEntry* e = d.entries + (t % d.capacity);
    int first, last, n, slot;
    asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(first) : "l"(&e->first_prog) : "memory");
    asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(last) : "l"(&e->last_prog) : "memory");
    asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(n) : "l"(&e->n_qubits) : "memory");
    asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(slot) : "l"(&e->slot) : "memory");
    double result = 0.0;
    run_small_request<R>(progs, first, last, n, s, red, s_result);
    if (threadIdx.x == 0) {
      result = s_result;
      d.results[slot] = result;
      __threadfence_system();  // the result is visible before the done word (also a release store)
      asm volatile("st.release.sys.global.s64 [%0], %1;" ::"l"(d.done + slot), "l"(t + 1) : "memory");
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

// ---- TMA pass: tensor maps and launch

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link-time dependency on libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return (EncodeTiledFn)p;
  }();
  return fn;
}

// The five-dimensional map of one pass (see k_sweep_tma) and its box
// geometry; false when this pass's tile cannot be described that way.
template <typename R>
static bool tma_map_for(Cx<R>* state, const ProgramHeader& h, CUtensorMap& map, TmaBoxes& bx) {
  constexpr int E = sizeof(Cx<R>) == 8 ? 4 : 3;  // 2^E amplitudes per 128-byte row
  if (h.m < E + 4 || h.L < E + 1 || h.m - (E + 4) > 5 || h.n <= h.m) return false;
  if ((uintptr_t)state % 256) return false;
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  bx.q1 = h.tq[E + 1];
  bx.q2 = h.tq[E + 2];
  bx.q3 = h.tq[E + 3];
  bx.nhq = h.m - (E + 4);
  for (int i = 0; i < kMaxTileQ; i++) bx.hq[i] = i < bx.nhq ? h.tq[E + 4 + i] : 0;
  const cuuint64_t amp = sizeof(Cx<R>);
  const cuuint64_t dims[5] = {128 / sizeof(R), 1ull << (bx.q1 - E), 1ull << (bx.q2 - bx.q1),
                              1ull << (bx.q3 - bx.q2), 1ull << (h.n - bx.q3)};
  const cuuint64_t strides[4] = {128, amp << bx.q1, amp << bx.q2, amp << bx.q3};
  const cuuint32_t box[5] = {(cuuint32_t)(128 / sizeof(R)), 2, 2, 2, 2};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(&map, sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5,
                         (void*)state, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Groups of the TMA pass (tiles in work at once per SM): four of 128 threads
// hold the SM's register file at 128 registers a thread.  Measured on the
// 28-qubit layered circuit: three groups 1.65 ms per pass, four 1.44.
constexpr int kTmaGroups = 4;
// Shared memory of a TMA pass with ns stages.
template <typename R>
static size_t tma_smem_bytes(const ProgramHeader& h, int ns) {
  return 1024 + (size_t)ns * (sizeof(Cx<R>) << h.m) + sizeof(Cx<R>) * (size_t)((h.ncoef + 1) & ~1) +
         16 * (size_t)kTmaMaxStages + 16 + 32 + 16 * 32;
}

template <typename R, int KMAX, int RQ, int OPS>
static cudaError_t launch_sweep_tma_k(Cx<R>* state, const SweepProgram<R>& prog, const CUtensorMap& map,
                                      const TmaBoxes& bx, cudaStream_t stream) {
  constexpr int NC = kTmaGroups;
  int ns = kTmaMaxStages;  // as many stages as shared memory holds
  while (ns > NC && tma_smem_bytes<R>(prog.h, ns) > 227 * 1024) ns--;
  if (ns <= NC) return cudaErrorInvalidConfiguration;
  const size_t smem = tma_smem_bytes<R>(prog.h, ns);
  static size_t configured_bytes[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem > configured_bytes[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_tma<R, KMAX, RQ, OPS, NC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured_bytes[dev] = smem;
  }
  const uint64_t ntiles = 1ull << (prog.h.n - prog.h.m);
  uint64_t grid = (uint64_t)device_sm_count();
  if (grid > ntiles) grid = ntiles;
  k_sweep_tma<R, KMAX, RQ, OPS, NC>
      <<<(unsigned)grid, NC * tma_group_threads<RQ>(), smem, stream>>>(state, map, bx, prog, ns);
  return cudaGetLastError();
}

// Whether the TMA pass runs this program: complex64 states of at least 2^9
// tiles whose tile groups are 128 threads (12-qubit tiles with five register
// qubits), unless a serving session is live on the device or SV_SWEEP_TMA=0
// in the environment selects the cp.async kernel.  (complex128 passes are bound by the FP64 pipe, and at the 128
// registers of four 128-thread groups per SM their register phases spill.)
static std::atomic<int> g_live_sessions[64];

void session_opened(int device) {
  if (device >= 0 && device < 64) g_live_sessions[device]++;
}
void session_closed(int device) {
  if (device >= 0 && device < 64) g_live_sessions[device]--;
}
bool session_live(int device) { return device >= 0 && device < 64 && g_live_sessions[device].load() > 0; }

static bool tma_enabled() {
  const char* e = std::getenv("SV_SWEEP_TMA");
  if (e && e[0] == '0') return false;
  int dev = 0;
  cudaGetDevice(&dev);
  return !session_live(dev);
}

template <typename R, int RQ>
static cudaError_t launch_sweep_tma(Cx<R>* state, const SweepProgram<R>& prog, cudaStream_t stream, bool& used) {
  used = false;
  if (!tma_enabled() || prog.h.n - prog.h.m < 9 || (1 << (prog.h.m - RQ)) != tma_group_threads<RQ>())
    return cudaSuccess;
  CUtensorMap map;
  TmaBoxes bx;
  if (!tma_map_for<R>(state, prog.h, map, bx)) return cudaSuccess;
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
  used = true;
  if (kmax <= 2 && !other) {
    if (!perm) return launch_sweep_tma_k<R, 2, RQ, kOpsRot>(state, prog, map, bx, stream);
    return launch_sweep_tma_k<R, 2, RQ, kOpsPerm>(state, prog, map, bx, stream);
  }
  if (kmax <= 2) return launch_sweep_tma_k<R, 2, RQ, kOpsAll>(state, prog, map, bx, stream);
  if (kmax == 3) return launch_sweep_tma_k<R, 3, RQ, kOpsAll>(state, prog, map, bx, stream);
  return launch_sweep_tma_k<R, 5, RQ, kOpsAll>(state, prog, map, bx, stream);
}

template <typename R>
cudaError_t launch_sweep(Cx<R>* state, const SweepProgram<R>& prog, cudaStream_t stream, const char** kernel) {
  // four register qubits with two tile buffers, or five with one (12-qubit
  // complex64 tiles; complex128 tiles have 11 qubits); large complex64 states
  // take the TMA pass
  bool used = false;
  if (kernel) *kernel = "sweep";
  if constexpr (sizeof(R) == 4) {
    if (prog.h.rq == 5) {
      cudaError_t e = launch_sweep_tma<R, 5>(state, prog, stream, used);
      if (used && kernel) *kernel = "sweep_tma";
      if (used || e != cudaSuccess) return e;
      return launch_sweep_rq<R, 5, SV_RQ5_DBUF>(state, prog, stream);
    }
  }
  if (prog.h.rq != 4) return cudaErrorInvalidValue;
  return launch_sweep_rq<R, 4, true>(state, prog, stream);
}

// Reads and clears the status a pass kernel recorded (SV_OK if none); the
// caller has synchronized the work it wants covered.
int take_sweep_status(cudaStream_t stream) {
  int st = 0, zero = 0;
  if (cudaMemcpyFromSymbolAsync(&st, g_sweep_status, sizeof(int), 0, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess) {
    cudaGetLastError();
    return (int)SV_ERR_CUDA;
  }
  if (st != 0) {
    cudaMemcpyToSymbolAsync(g_sweep_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, stream);
    cudaStreamSynchronize(stream);
  }
  return st;
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

template <typename R>
cudaError_t launch_small_session(const SmallSessionDev& d, const SweepProgram<R>* progs, int max_n, int grid,
                                 cudaStream_t stream) {
  const int smem = (int)sizeof(Cx<R>) << max_n;
  static int configured_bytes[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem > 48 * 1024 && smem > configured_bytes[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_small_session<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured_bytes[dev] = smem;
  }
  k_small_session<R><<<grid, 256, smem, stream>>>(d, progs);
  return cudaGetLastError();
}

template cudaError_t launch_small_session<float>(const SmallSessionDev&, const SweepProgram<float>*, int, int,
                                                 cudaStream_t);
template cudaError_t launch_small_session<double>(const SmallSessionDev&, const SweepProgram<double>*, int, int,
                                                  cudaStream_t);
template cudaError_t launch_small_batch<float>(const SweepProgram<float>*, const int*, const int*, int, int, double*,
                                               cudaStream_t);
template cudaError_t launch_small_batch<double>(const SweepProgram<double>*, const int*, const int*, int, int, double*,
                                                cudaStream_t);
template cudaError_t launch_sweep<float>(Cx<float>*, const SweepProgram<float>&, cudaStream_t, const char**);
template cudaError_t launch_sweep<double>(Cx<double>*, const SweepProgram<double>&, cudaStream_t, const char**);
template cudaError_t launch_init_basis<float>(Cx<float>*, int, uint64_t, cudaStream_t);
template cudaError_t launch_init_basis<double>(Cx<double>*, int, uint64_t, cudaStream_t);

}  // namespace sv
