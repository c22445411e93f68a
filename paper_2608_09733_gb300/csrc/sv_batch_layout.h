// sv_batch_layout.h -- the batched program of one adjoint pass: the structures
// the host builder (sv_adjoint_host.cpp) writes and the batched sweep kernels
// read, both the library's interpreting kernel (sv_adjoint.cu) and the kernels
// compiled at run time from one program (sv_jit_batch.cpp).  No host headers.
#pragma once

#include "sv_prog_layout.h"

namespace sv {

// BOp.flags only (batched programs): the op's matrix is real, and the
// generator of a parameterised one-qubit rotation is X, Y or Z (closed-form
// gradient terms).
constexpr uint16_t OPF_REALM = 8;
constexpr uint16_t OPF_GX = 16;
constexpr uint16_t OPF_GY = 32;
constexpr uint16_t OPF_GZ = 64;

// ----------------------------------------------------------------- batched programs
//
// The adjoint gradient runs B states of one circuit template side by side
// (Sec. 4.1 BatchSV: a batch of states evolved together; parameter values
// differ per state).  A batched op takes its coefficients either from the
// program pool (constant gates) or from a per-state table built on the host in
// double precision (parameterised gates).  In reverse mode each op first adds
// Im <lambda|G|psi> over the tile (G the gate's generator, with its control
// projector) and then applies the conjugate transpose to psi and lambda.

struct BOp {
  uint8_t kind;         // OPK_DENSE / OPK_DIAG / OPK_ANTIDIAG / OPK_SWAP / OPK_SIGN, k <= 2
  uint8_t k;
  uint8_t pos[2];       // local positions (matrix order); OPK_DIAG: 0xFF = external
  uint8_t spos[2];      // sorted local positions
  uint8_t gq[2];        // global qubits (OPK_DIAG external bits)
  uint8_t rs[2];        // register slots in a register phase (0xFF: none)
  uint8_t table;        // 1: coefficients from the per-state table row `coef`
  uint8_t dagger;       // 1: apply the conjugate transpose
  uint8_t grad;         // 1: accumulate Im <lambda|G|psi> into gradient `gidx`
  uint8_t gacc;         // local accumulator index of a gradient op
  uint8_t rmask, rval;  // controls on register slots (register phase)
  uint32_t lmask, lval; // all local controls (shared-memory phase)
  uint32_t tmask, tval; // local controls held by the thread index (register phase)
  uint64_t xmask, xval;
  uint32_t coef;        // pool offset, or table row when `table`
  uint32_t gen;         // pool offset of the generator (d x d dense, or d diagonal entries)
  uint32_t gidx;        // index of the parameterised gate (gradient scratch row)
  uint16_t flags;       // OPF_* flags
  uint16_t soff;        // offset of the op's matrix (then its generator) in the CTA's shared copy
};
static_assert(sizeof(BOp) == 64, "BOp layout");

constexpr int kBatchOps = 96;
constexpr int kBatchGacc = 64;   // gradient accumulators per program
constexpr int kTableStride = 16; // complex entries per (gate, state) table row

struct BatchHeader {
  int32_t n, m, L, nops;
  int32_t batch, ngacc, ngrad_total, nphases;
  int32_t scoef, pad;  // complex entries of the shared coefficient copy
  int8_t tq[16];
};

template <typename R>
struct BatchProgram {
  static constexpr int kPool = (kProgramBytes - (int)sizeof(BatchHeader) - kBatchOps * (int)sizeof(BOp) -
                                kMaxPhases * (int)sizeof(Phase)) /
                               (int)sizeof(Cx<R>);
  BatchHeader h;
  BOp ops[kBatchOps];
  Phase ph[kMaxPhases];
  Cx<R> pool[kPool];
};

}  // namespace sv
