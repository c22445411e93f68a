// sv_prog_layout.h -- the device program of one pass: the structures the
// host program builder (sv_program.cpp) writes and the pass kernels read,
// both the library's interpreting kernel (sv_sweep.cu) and the kernels
// compiled at run time from one program (sv_jit.cpp).  No host headers, so
// the run-time compiler takes it as it is.
#pragma once

#ifdef __CUDACC_RTC__
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef int int32_t;
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
#else
#include <stdint.h>
#endif

namespace sv {

// ----------------------------------------------------------------- device program
//
// One "sweep" = one pass over the state in tiles of 2^m amplitudes.  A tile is
// the set of amplitudes that share the bits outside the tile qubits tq[0..m-1]
// (ascending; tq[i] == i for i < L so each tile is made of contiguous runs of
// 2^L amplitudes).  The kernel gathers a tile into shared memory, applies the
// program's ops in order, and scatters it back.  An op acts on *local* bit
// positions (indices into tq); control qubits outside the tile are the same for
// every amplitude of a tile and are tested once per tile.

enum OpKind : uint8_t {
  OPK_DENSE = 0,    // dense 2^k x 2^k complex matrix on local positions pos[0..k-1]
  OPK_REAL = 1,     // dense matrix with all-real entries (k <= 2)
  OPK_DIAG = 2,     // diagonal 2^k entries; the k bits may be local or external
  OPK_ANTIDIAG = 3, // one qubit: out0 = a * v1, out1 = b * v0 (X, Y, CNOT ...)
  OPK_SWAP = 4,     // two local positions: exchange |01> and |10>
  OPK_SIGN = 5,     // negate the amplitudes whose bits match (CZ, Z, CCZ ...): no coefficients
  OPK_KRON = 6,     // register phase only: uncontrolled 2x2 matrices on register slots (rmask = the
                    // slots present), four blocks of four coefficients at `coef`
  OPK_KROT = 7,     // register phase only: real rotations [[C, -S], [S, C]] on register slots (rmask =
                    // the slots present).  complex64: three shears, coef[s] = (tan(alpha/2), sin(alpha));
                    // complex128: scaled form, coef[s].re = S/C (bit s of rval clear) or C/S (set), the
                    // factor max(C, S) carried by a phase table
  OPK_PHASE = 8,    // register phase only: amplitude j of the thread's 2^RQ is multiplied by
                    // coef[var * table_stride(RQ) + j]; var collects k selector bits, selector i being bit
                    // gq[i] of the thread's local bits (gq[i] < 64) or global bit gq[i] - 64 of the tile
};

// DevOp.pad flag bits
constexpr uint8_t OPF_FLIP = 1;   // anti-diagonal (1, 1): a pure bit flip
constexpr uint8_t OPF_TCOND = 2;  // tmask/tval is not empty
constexpr uint8_t OPF_XCOND = 4;  // xmask/xval is not empty

// In a register phase DevOp.pad holds the op's dispatch word, so one load
// decides what to do: kind | flags << 4 | rmask << 7 | rval << 12 | coef << 17
// (OPK_SIGN: the pattern stays in DevOp.coef and the coef field is 0).
constexpr uint32_t op_code(uint32_t kind, uint32_t flags, uint32_t rmask, uint32_t rval, uint32_t coef) {
  return kind | (flags << 4) | (rmask << 7) | (rval << 12) | (coef << 17);
}
constexpr int kCodeCoefMax = 1 << 15;

// Entries between the variants of a phase table: 2^rq plus padding so that
// variants start in different shared-memory banks and (complex64) stay
// 16-byte aligned for pairwise loads.
template <typename R>
constexpr int table_stride(int rq) {
  return (1 << rq) + (sizeof(R) == 4 ? 2 : 1);
}

constexpr int kMaxTileQ = 14;  // 2^14 amplitudes: 128 KiB (c64) of shared memory
constexpr int kMaxOps = 96;
constexpr int kMaxPhases = 96;
constexpr int kRegQ = 4;        // register qubits of a phase (default: 16 amplitudes per thread)
constexpr int kMaxRegQ = 5;     // at most 32 amplitudes per thread
constexpr int kProgramBytes = 32000;  // kernel parameter space is 32764 bytes

// An op as the kernel sees it.  Positions are local tile bits (indices into
// tq).  In a register phase, rs[] gives the register slot of each matrix bit
// (0xFF: not in registers), and the controls are split into the register part
// (rmask/rval over slots), the thread part (tmask/tval over local bits held by
// the thread index) and the part outside the tile (xmask/xval, global bits).
struct DevOp {
  uint8_t kind;
  uint8_t k;            // matrix qubits
  uint8_t pos[5];       // local positions, matrix order (pos[0] = least significant matrix bit);
                        // OPK_DIAG/OPK_SIGN: 0xFF marks an external qubit (see gq)
  uint8_t spos[5];      // the local positions sorted ascending (group enumeration)
  uint8_t gq[5];        // global qubit of each matrix bit
  uint8_t rs[5];        // register slot of each matrix bit in its phase, 0xFF if none
  uint8_t rmask, rval;  // control bits on register slots
  uint32_t lmask, lval; // all local controls (shared-memory path)
  uint32_t tmask, tval; // local controls held by the thread index (register path)
  uint64_t xmask, xval; // controls outside the tile (global bit mask / required values)
  uint32_t coef;        // first coefficient in the program's pool (OPK_SIGN in a register
                        // phase: the 16-bit pattern of register combinations to negate)
  uint32_t pad;         // OPF_* flags
};
static_assert(sizeof(DevOp) == 64, "DevOp layout");

enum PhaseKind : uint8_t { PH_REG = 0, PH_SMEM = 1 };

// A run of ops applied with the same amplitude-to-thread mapping.  PH_REG:
// thread t holds the 16 amplitudes whose local bits at rp[] vary and whose
// other local bits are t deposited into tpos[] (ascending); PH_SMEM: one op
// applied group by group straight in shared memory (dense k >= 3 and wide
// diagonals).
struct Phase {
  uint8_t kind, first, nops, ntpos, nrp;
  uint8_t rp[kMaxRegQ];
  uint8_t tpos[kMaxTileQ];
};
static_assert(sizeof(Phase) == 24, "Phase layout");

template <typename R>
struct Cx {
  R re, im;
};

struct ProgramHeader {
  int32_t n, m, L, nops;
  int32_t ncoef, nphases;
  int32_t rq, pad;  // register qubits of the register phases (4 or 5)
  int8_t tq[16];
};

template <typename R>
struct SweepProgram {
  static constexpr int kPool = (kProgramBytes - (int)sizeof(ProgramHeader) - kMaxOps * (int)sizeof(DevOp) -
                                kMaxPhases * (int)sizeof(Phase)) /
                               (int)sizeof(Cx<R>);
  ProgramHeader h;
  DevOp ops[kMaxOps];
  Phase ph[kMaxPhases];
  Cx<R> coef[kPool];
};
static_assert(sizeof(SweepProgram<float>) % 16 == 0 && sizeof(SweepProgram<double>) % 16 == 0,
              "programs in an array keep 16-byte alignment");

}  // namespace sv
