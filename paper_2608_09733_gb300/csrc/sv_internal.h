// sv_internal.h -- structures shared by the host planner (sv_plan.cpp, sv_api.cpp)
// and the CUDA kernels (sv_sweep.cu, sv_reduce.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "sv_prog_layout.h"

namespace sv {

using cplx = std::complex<double>;

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

// *kernel (if not NULL) names the pass kernel that ran: "sweep_jit" (the
// program's own compiled kernel, TMA tile movement), "sweep_tma" (TMA, the
// interpreting kernel) or "sweep" (cp.async).  jit (if not NULL) is the
// program's compiled kernel, used wherever the TMA pass runs.
struct JitKernel;
template <typename R>
cudaError_t launch_sweep(Cx<R>* state, const SweepProgram<R>& prog, cudaStream_t stream,
                         const char** kernel = nullptr, const JitKernel* jit = nullptr);
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
// Live sessions per device and their resident CTAs.  A session's CTAs hold
// their SMs, so while one is live the TMA pass (one CTA per SM, a fixed share
// of tiles each) launches on the SMs the sessions leave free.
void session_opened(int device, int ctas);
void session_closed(int device, int ctas);
bool session_live(int device);
// Ends the kernels of the device's live sessions and holds them (their locks)
// until sessions_release, which relaunches those with requests not done
// (sv_serve.cpp): a module load waits for every resident kernel to end.
void sessions_quiesce(int device, std::vector<sv_small_session*>& held);
void sessions_release(std::vector<sv_small_session*>& held);

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

// ----------------------------------------------------------------- run-time compiled pass kernels
// (sv_jit.cpp).  jit_mode(): 0 off, 1 compile a program structure on its
// second use, 2 on its first (SV_JIT=0 / 1 / 2 in the environment, or
// jit_set_mode; -1 goes back to the environment).
int jit_mode();
void jit_set_mode(int mode);
// The kernel source of one program, empty if the TMA pass would not run it.
template <typename R>
std::string jit_source(const SweepProgram<R>& P);
// Compiled kernels for a circuit's programs (NULL entries: the interpreting
// kernel runs that pass); compiles what the cache lacks, in parallel.
template <typename R>
std::vector<const JitKernel*> jit_compile_programs(const std::vector<SweepProgram<R>>& progs);
// A program's structure key (empty if the TMA pass would not run it): all its
// kernel source is written from, none of its coefficient values.
std::string jit_program_key(const SweepProgram<float>& P);
// The programs' kernels by structure key: counts a use of each key, compiles
// (in the calling thread, in parallel) the keys used at least `threshold`
// times that have no kernel yet; NULL entries interpret.
std::vector<const JitKernel*> jit_program_kernels(const std::vector<SweepProgram<float>>& progs,
                                                  const std::vector<std::string>& keys, int threshold);
// Launches a compiled pass kernel with the interpreting TMA kernel's
// arguments (map: the CUtensorMap, bx: the TmaBoxes).
cudaError_t jit_launch(const JitKernel* k, void* state, const void* map, const void* bx, const void* prog, int ns,
                       int* status, unsigned grid, unsigned block, size_t smem, cudaStream_t stream);
// Generates (and with compile, compiles for sm_<arch>a) every program's kernel
// without a device.
template <typename R>
void jit_check_programs(const std::vector<SweepProgram<R>>& progs, bool compile, int arch, int* n_sources,
                        int* n_compiled, std::string* first_error, std::string* sources);
void jit_stats(long long* compiled, long long* failed, long long* launches, double* compile_seconds,
               std::string* last_error);
bool jit_available(std::string* why);

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
