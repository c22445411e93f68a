// sv_adjoint.h -- structures and launch declarations of the batched adjoint
// kernels (sv_adjoint.cu, sv_adjoint_host.cpp).  Not part of the public ABI;
// kept apart from sv_internal.h so the pass kernel's sources do not depend
// on them.
#pragma once

#include "sv_internal.h"
#include "sv_batch_layout.h"

namespace sv {

// Batched kernels (sv_adjoint.cu).  psi/lam hold `batch` states of 2^n
// amplitudes back to back.  `table` is [gates][batch][kTableStride].
// jit (if not NULL): the program's compiled kernel (sv_jit.cpp), launched in
// place of the interpreting one with the same arguments.
template <typename R>
cudaError_t launch_batch_sweep(Cx<R>* psi, Cx<R>* lam, const Cx<R>* table, double* gscratch, int grid_x,
                               const BatchProgram<R>& prog, bool reverse, cudaStream_t stream,
                               const JitKernel* jit = nullptr);
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
// ----------------------------------------------------------------- compiled batched kernels (sv_jit.cpp)
// The kernel source of one batched program (every phase and op a constant).
template <typename R>
std::string jit_batch_source(const BatchProgram<R>& P, bool rev);
// Compiles (in parallel, what the cache lacks) the kernels of these programs
// and records them by program for jit_batch_lookup.
template <typename R>
void jit_batch_prepare(const std::vector<const BatchProgram<R>*>& progs, const std::vector<char>& rev);
// The compiled kernel of a program prepared before on this device, or NULL.
template <typename R>
const JitKernel* jit_batch_lookup(const BatchProgram<R>& P, bool rev);
cudaError_t jit_batch_launch(const JitKernel* k, void* psi, void* lam, const void* table, double* gscratch,
                             const void* prog, unsigned grid_x, unsigned batch, unsigned threads, size_t smem,
                             cudaStream_t stream);
// Writes (and with compile, compiles for sm_<arch>a) the distinct kernels of
// these programs without a device.
template <typename R>
void jit_check_batch(const std::vector<const BatchProgram<R>*>& progs, const std::vector<char>& rev, bool compile,
                     int arch, int* n_sources, int* n_compiled, std::string* first_error, std::string* sources);
}  // namespace sv
