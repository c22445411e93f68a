// sv_internal.h -- structures shared by the host planner (sv_plan.cpp, sv_api.cpp)
// and the CUDA kernels (sv_sweep.cu, sv_reduce.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "../../include/sv.h"

namespace sv {

using cplx = std::complex<double>;

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


// ----------------------------------------------------------------- host plan

// A gate after lowering (a matrix in double precision) or a fused block.
struct LOp {
  OpKind kind = OPK_DENSE;
  int k = 0;                 // matrix qubits
  int q[5] = {0, 0, 0, 0, 0};  // global matrix qubits, q[0] = least significant matrix bit
  int nc = 0;
  int c[5] = {0, 0, 0, 0, 0};  // global control qubits
  int cs[5] = {1, 1, 1, 1, 1}; // required control states
  std::vector<cplx> m;       // DENSE/REAL: 2^k x 2^k row-major; DIAG: 2^k; ANTIDIAG: {a, b}
  uint64_t touch = 0;        // every qubit the op reads (matrix qubits and controls)
  uint64_t need = 0;         // qubits that must be inside the tile
  int first_gate = 0;        // index of the first source gate (fusion bookkeeping)
};

struct Sweep {
  int m = 0, L = 0;
  int tq[kMaxTileQ];
  std::vector<int> ops;      // indices into the LOp list, in application order
};

struct Plan {
  int n = 0;
  std::vector<LOp> ops;
  std::vector<int> block_starts;  // first gate of each op (fusion blocks) + n_gates
  std::vector<Sweep> sweeps;
};

// Errors carry a status and a message up to the C ABI.
struct Error {
  sv_status status;
  std::string msg;
};

[[noreturn]] inline void fail(sv_status s, const std::string& m) { throw Error{s, m}; }
inline void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(SV_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
void set_last_error(const std::string& m);

// Runs f, mapping sv::Error and host exceptions to an sv_status.
template <typename F>
sv_status guarded(F&& f) {
  try {
    f();
    return SV_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.status;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return SV_ERR_OOM;
  } catch (...) {
    set_last_error("unexpected host exception");
    return SV_ERR_INVALID;
  }
}

// Device pointer checks (device/managed memory of the current device, 16-byte
// aligned, inside its allocation) and library-owned scratch: one grow-only
// buffer per (device, stream, name).
void check_device_buffer(const void* p, size_t bytes, const char* what);
void* scratch_buffer(cudaStream_t stream, const char* name, size_t bytes);

// Pinned host staging per (device, stream, name), grow-only; `ready` is
// recorded after the last copy out of it, so a rewrite waits for that copy.
struct Pinned {
  void* p = nullptr;
  size_t cap = 0;
  cudaEvent_t ready = nullptr;
};
Pinned& pinned_buffer(cudaStream_t stream, const char* name, size_t bytes);

// Lowering (gate records -> double-precision matrices), the paper's greedy
// fusion, and the tile scheduler.  Throw sv::Error on invalid input.
void validate_gates(int n, const sv_gate* gates, size_t n_gates, size_t n_param_values);
std::vector<cplx> gate_matrix(const sv_gate& g, const double* param_values);
LOp lower_gate(const sv_gate& g, const double* param_values, int index);
std::vector<LOp> fuse_greedy(int n, const sv_gate* gates, size_t n_gates, const double* param_values, int kmax,
                             std::vector<int>* block_starts, bool dense_always);
void classify(LOp& op);
std::vector<Sweep> schedule_sweeps(int n, const std::vector<LOp>& ops, int tile_q, int low_q, int coef_pool,
                                   int ops_per_pass);
Plan make_plan(int n, sv_dtype dtype, const sv_gate* gates, size_t n_gates, const double* param_values,
               size_t n_param_values, const sv_exec_opts& opts, int tile_q_override = 0);
double op_cost(const LOp& op);
int tile_qubits_for(sv_dtype dtype, int n);
int low_qubits_for(sv_dtype dtype);
int reg_qubits_for(int m);  // register qubits of a tile of m qubits (4, or 5 for m >= 12)

// The kernel program of one sweep (sv_program.cpp); rq_override > 0 forces the
// register qubits of the register phases.
// A 2x2 unitary U written as g * diag(1, ephi) * [[C, -S], [S, C]] * diag(1, elam)
// (the Z-Y-Z Euler form, C = cos(alpha), S = sin(alpha), alpha in [0, pi/2]);
// false if the reconstruction misses U by more than tol in any entry.
struct RotSplit {
  cplx g = 1.0, ephi = 1.0, elam = 1.0;
  double C = 1.0, S = 0.0;
};
bool rot_split(const cplx* U, double tol, RotSplit& r);

template <typename R>
void build_program(const Plan& plan, const Sweep& sw, SweepProgram<R>& P, int rq_override = 0);

// ----------------------------------------------------------------- launches
// (sv_sweep.cu / sv_reduce.cu).  All return cudaError_t of the launch.

// *kernel (if not NULL) names the pass kernel that ran: "sweep_tma" (TMA
// tile movement) or "sweep" (cp.async).
template <typename R>
cudaError_t launch_sweep(Cx<R>* state, const SweepProgram<R>& prog, cudaStream_t stream,
                         const char** kernel = nullptr);
template <typename R>
cudaError_t launch_init_basis(Cx<R>* state, int n, uint64_t index, cudaStream_t stream);
// One CTA per small request (whole state in shared memory): request b runs
// programs first_prog[b] .. first_prog[b+1]-1 and writes sum_q <Z_q> to out[b].
template <typename R>
cudaError_t launch_small_batch(const SweepProgram<R>* progs, const int* first_prog, const int* nq, int n_requests,
                               int max_n, double* out, cudaStream_t stream);

// Persistent packed small states (serving sessions, sv_serve.cpp).  The
// entries, published count, exit flag, results and done words are pinned host
// memory mapped into the device; head and status are device memory.
struct SmallEntry {
  int32_t first_prog, last_prog;  // the request's programs in the session's program arena
  int32_t n_qubits, slot;         // state size; result slot (results[slot], done[slot])
};
struct SmallSessionDev {
  const SmallEntry* entries;      // ring of `capacity` entries; ticket t uses entries[t % capacity]
  const long long* tail;          // tickets published so far (written by the host)
  const int* exit_flag;           // nonzero: end the session once no published ticket is left
  unsigned long long* head;       // next ticket to claim (device)
  double* results;                // sum_q <Z_q> per slot
  long long* done;                // done[slot] = ticket + 1 once results[slot] is written
  int* status;                    // SV_OK, or SV_ERR_TIMEOUT when a wait ran out (device)
  long long capacity;
  uint64_t limit_ns;              // longest wait for a ticket
};
template <typename R>
cudaError_t launch_small_session(const SmallSessionDev& d, const SweepProgram<R>* progs, int max_n, int grid,
                                 cudaStream_t stream);
// Live sessions per device.  A session's resident CTAs hold their SMs, so
// while one is live the pass kernels avoid the TMA kernel (one CTA per SM, a
// fixed share of tiles each) for the cp.async one, whose many small CTAs fill
// what the session leaves free.
void session_opened(int device);
void session_closed(int device);
bool session_live(int device);

// Reductions write fixed-order per-block partials into `scratch` and a final
// kernel folds them into `out` (device doubles).
template <typename R>
cudaError_t launch_expect_z_all(const Cx<R>* state, int n, double* scratch, size_t scratch_doubles, double* out,
                                cudaStream_t stream);
template <typename R>
cudaError_t launch_expect_terms(const Cx<R>* state, int n, const sv_pauli_term* terms, int n_terms, double* scratch,
                                size_t scratch_doubles, double* out, cudaStream_t stream);
size_t expect_z_all_scratch_doubles(int n);

size_t expect_terms_scratch_doubles(int n, int n_terms);

int device_sm_count();

// Reads and clears the status a pass kernel recorded on the device (SV_OK, or
// SV_ERR_TIMEOUT when a bounded wait ran out); synchronizes `stream`.
int take_sweep_status(cudaStream_t stream);

// Kernel timing (sv_profile_*): Prof p(stream, "sweep", bytes); launch; p.done();
struct Prof {
  Prof(cudaStream_t s, const char* family, double bytes);
  void done();
  cudaStream_t stream;
  const char* family;
  double bytes;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

}  // namespace sv
