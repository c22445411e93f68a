// sv_adjoint.h -- structures and launch declarations of the batched adjoint
// kernels (sv_adjoint.cu, sv_adjoint_host.cpp).  Not part of the public ABI;
// kept apart from sv_internal.h so the pass kernel's sources do not depend
// on them.
#pragma once

#include "sv_internal.h"

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

// Batched kernels (sv_adjoint.cu).  psi/lam hold `batch` states of 2^n
// amplitudes back to back.  `table` is [gates][batch][kTableStride].
template <typename R>
cudaError_t launch_batch_sweep(Cx<R>* psi, Cx<R>* lam, const Cx<R>* table, double* gscratch, int grid_x,
                               const BatchProgram<R>& prog, bool reverse, cudaStream_t stream);
int batch_grid_x(int n, int m, int batch);
template <typename R>
cudaError_t launch_batch_init(Cx<R>* psi, int n, int batch, cudaStream_t stream);
// lam (=|+=) sum_j c_j P_j psi over the terms sharing one x mask
template <typename R>
cudaError_t launch_pauli_accum(const Cx<R>* psi, Cx<R>* lam, int n, int batch, uint64_t x, const uint64_t* z,
                               const double* c, int nt, bool accumulate, cudaStream_t stream);
// lam (+)= sum_j c_j P_j psi over the batch, in tiles that hold whole X-masks;
// with `row_coeffs` (device, batch x n_terms) state b uses c_{b,j} (then every
// X-mask must fit a tile, else cudaErrorNotSupported).
template <typename R>
cudaError_t launch_pauli_tiles(const Cx<R>* psi, Cx<R>* lam, int n, int batch, const sv_pauli_term* terms,
                               int n_terms, bool accumulate, const double* row_coeffs, cudaStream_t stream);
// out[b] = Re <psi_b|lam_b> (partials in scratch: batch x grid doubles)
template <typename R>
cudaError_t launch_batch_dot(const Cx<R>* psi, const Cx<R>* lam, int n, int batch, double* scratch, double* out,
                             cudaStream_t stream);
size_t batch_dot_scratch_doubles(int batch);
// out[b * ngrad + g] = sum over grid_x of gscratch[(b * ngrad + g) * grid_x + c]
cudaError_t launch_grad_finish(const double* gscratch, int batch, int ngrad, int grid_x, double* out,
                               cudaStream_t stream);

// A parameterised gate of a template, for tables built on the device: its
// family (one-parameter rotation) and the parameter slot it reads.
struct TableGate {
  int32_t type;
  int32_t slot;
};
// table[(g * batch + b) * kTableStride ..] = the matrix of gate g at
// params[b * npar + gates[g].slot] (device arrays), as the host would build it.
template <typename R>
cudaError_t launch_build_tables(const double* params, int npar, int batch, const TableGate* gates, int ngates,
                                Cx<R>* table, cudaStream_t stream);
// out[b * npar + p] = sum over k with slot[k] == p of g[b * ngrad + k] (device).
cudaError_t launch_scatter_grad(const double* g, int batch, int ngrad, const int* slot, int npar, double* out,
                                cudaStream_t stream);
}  // namespace sv
