/*
 * sv.h -- C ABI of the GB300 state-vector library (libsv.so).
 *
 * The library applies quantum circuits to a dense state vector of 2^n complex
 * amplitudes held in device memory, evaluates Pauli-string expectations and
 * computes adjoint gradients.  It is the hot path of the state-vector engine of
 * "Aicir: A Full-Stack Quantum Circuit Simulator with Ascend NPU Support":
 * circuits are given as the paper states them (Sec. 4.2: gate family, target
 * qubits before control qubits, optional control states, parameters bound from
 * a shared vector), Hamiltonians as weighted Pauli strings (Sec. 4.2, Sec. 4.4).
 *
 * Conventions
 *   - Qubit q is bit q of the basis index (little-endian).  For a k-qubit
 *     matrix, targets[0] is the least significant bit of its row/column index.
 *   - Rotations are R_P(theta) = exp(-i theta P / 2) (Sec. 9.1).
 *   - U3(th, ph, la) = [[cos(th/2), -e^{i la} sin(th/2)],
 *                       [e^{i ph} sin(th/2), e^{i(ph+la)} cos(th/2)]],
 *     U2(ph, la) = U3(pi/2, ph, la), P(la) = diag(1, e^{i la}).
 *   - A state is 2^n amplitudes, interleaved (re, im): float pairs for SV_C64,
 *     double pairs for SV_C128, 16-byte aligned.  State memory belongs to the
 *     caller (e.g. a torch tensor); the library never frees it.
 *   - Gate matrices are built on the host in double precision and narrowed to
 *     the state's precision only when they are handed to the GPU (Sec. 3.3,
 *     Sec. 5.2).  Expectations and gradients are accumulated in double.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 *     return results in host memory synchronize that stream; all others only
 *     enqueue work on it.
 *
 * Errors (Sec. 3.3: unsupported combinations raise at the boundary)
 *   Every call validates its arguments before it touches the device and
 *   returns an sv_status; it never aborts the process.  sv_last_error() gives
 *   a message for the calling thread's last failure.  A failed call leaves
 *   device memory untouched unless the failure is SV_ERR_CUDA, which reports
 *   a CUDA runtime error (asynchronous errors surface at the next call that
 *   synchronizes).
 */
#ifndef SV_H
#define SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SV_OK = 0,
  SV_ERR_INVALID = 1,       /* bad argument: qubit out of range, repeated qubit, bad size ... */
  SV_ERR_UNSUPPORTED = 2,   /* valid request this library does not run (e.g. no generator) */
  SV_ERR_OOM = 3,           /* device allocation of library scratch failed */
  SV_ERR_CUDA = 4,          /* CUDA runtime error */
  SV_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out */
  SV_ERR_UNBOUND_PARAM = 6  /* a gate names a parameter slot that was not supplied (Sec. 4.2) */
} sv_status;

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype;

/* Gate families (Sec. 4.2 gate table).  Controlled forms (CX, CY, CZ, CRX,
 * CRY, CRZ, CCX, controlled phase ...) are the base family with
 * n_controls > 0.  The excitation families rotate the two basis states that
 * exchange one or two excitations and leave the rest alone, with
 * c = cos(theta/2), s = sin(theta/2) and i the matrix index:
 *   SV_GATE_EXC1 (single excitation / Givens, 2 targets): on i = 1, 2
 *     (|t0 t1> = |10>, |01>) the block [[c, -s], [s, c]];
 *   SV_GATE_EXC2 (double excitation, 4 targets): on i = 3, 12 (t0 t1 set,
 *     t2 t3 set) the same block.
 * Both are exp(-i theta G / 2) with G = Y on that pair of states and 0
 * elsewhere (spectrum {-1, 0, 1}, which is why the paper's shift rule for
 * them has four terms). */
typedef enum {
  SV_GATE_I = 0, SV_GATE_X, SV_GATE_Y, SV_GATE_Z, SV_GATE_H,
  SV_GATE_S, SV_GATE_SDG, SV_GATE_T, SV_GATE_TDG, SV_GATE_SX,
  SV_GATE_RX, SV_GATE_RY, SV_GATE_RZ, SV_GATE_P, SV_GATE_U2, SV_GATE_U3,
  SV_GATE_SWAP, SV_GATE_RXX, SV_GATE_RYY, SV_GATE_RZZ,
  SV_GATE_UNITARY,
  SV_GATE_EXC1, SV_GATE_EXC2,
  SV_GATE_COUNT_
} sv_gate_type;

#define SV_MAX_TARGETS 5
#define SV_MAX_CONTROLS 5
#define SV_MAX_QUBITS 34

/* One circuit operation (Sec. 4.2).
 *   type             sv_gate_type
 *   n_targets        1 for one-qubit families, 2 for SWAP/RXX/RYY/RZZ/EXC1,
 *                    4 for EXC2, 1..5 for SV_GATE_UNITARY
 *   targets          target qubits; targets[0] = least significant matrix bit
 *   n_controls       0..5 control qubits, distinct from the targets
 *   control_zero_mask bit j set: controls[j] enables the gate when it is |0>
 *                    (the paper's control state 0); clear: when it is |1>
 *   param_slot[i]    -1: angle i is params[i]; >= 0: angle i is
 *                    param_values[param_slot[i]] of the call (a shared
 *                    parameter vector); a slot beyond the supplied vector is
 *                    SV_ERR_UNBOUND_PARAM
 *   params           angles: RX/RY/RZ/P/RXX/RYY/RZZ/EXC1/EXC2 use params[0]; U2 uses
 *                    (phi, lambda); U3 uses (theta, phi, lambda)
 *   matrix           SV_GATE_UNITARY only: host pointer to 2^k x 2^k complex
 *                    entries, row-major, interleaved (re, im) doubles; read
 *                    during the call only (the caller keeps ownership) */
typedef struct sv_gate {
  int32_t type;
  int32_t n_targets;
  int32_t targets[SV_MAX_TARGETS];
  int32_t n_controls;
  int32_t controls[SV_MAX_CONTROLS];
  uint32_t control_zero_mask;
  int32_t param_slot[3];
  double params[3];
  const double* matrix;
} sv_gate;

/* A weighted Pauli string c * P with P|b> = i^{nY} (-1)^{popcount(b & z)}
 * |b xor x> (Sec. 4.4): bit q of x_mask/z_mask set means X/Z on qubit q, both
 * set means Y.  Bits at or above n_qubits are SV_ERR_INVALID. */
typedef struct sv_pauli_term {
  uint64_t x_mask;
  uint64_t z_mask;
  double coeff;
} sv_pauli_term;

/* Version of this ABI (major * 100 + minor). */
int sv_version(void);

/* Message for the calling thread's last failed call ("" if none).  The
 * pointer stays valid until the thread's next failing call. */
const char* sv_last_error(void);

/* Writes the basis state |basis_index> (Sec. 5.3: a run starts from
 * |0..0>) into `state` (device, 2^n amplitudes of dtype). */
sv_status sv_init_basis(void* state, int n_qubits, sv_dtype dtype, uint64_t basis_index, void* stream);

/* Applies the gates, in order, to `state` in place (Sec. 4.3 execution,
 * Sec. 5.3 gate application).
 *   state         device, 2^n amplitudes of dtype, modified in place
 *   gates         host array of n_gates records (read during the call)
 *   param_values  host array of n_param_values doubles bound to slots (may
 *                 be NULL when no gate uses a slot)
 *   fuse_max_k    0: no fusion; 2..5: the paper's fusion (Sec. 4.3 `fuse`,
 *                 Sec. 9.2): consecutive gates are joined, without changing
 *                 their order, into blocks of at most fuse_max_k qubits, each
 *                 applied as one dense 2^k x 2^k matrix; 1 or >5 is invalid.
 * Whatever the fusion setting, the library runs several consecutive gates or
 * blocks per pass over HBM when their qubits fit one shared-memory tile; the
 * order of operations on any qubit is never changed.
 * Enqueues kernels on `stream`; the call returns before they finish. */
sv_status sv_apply_circuit(void* state, int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                           const double* param_values, size_t n_param_values, int fuse_max_k, void* stream);

/* Execution options of sv_apply_circuit_ex.
 *   fuse_max_k      as in sv_apply_circuit (0, or 2..5)
 *   block_mode      SV_BLOCK_AUTO: a fused block runs as its dense 2^k x 2^k
 *                   matrix when that takes fewer multiply-adds per amplitude
 *                   than its gates, else as its gates inside the same pass
 *                   (identical up to rounding); SV_BLOCK_DENSE: every fused
 *                   block of two or more gates runs as its dense matrix, the
 *                   paper's form (Sec. 9.2)
 *   ops_per_pass    0: as many operations per pass over the state as fit a
 *                   tile; 1: one operation per pass (the plain per-gate path,
 *                   used as a baseline); other values cap the count
 *   tile_qubits     0: the library picks the tile width (the qubits a pass
 *                   gathers into shared memory) from the state size; 8..13
 *                   (complex64) or 8..11 (complex128) forces it (capped at
 *                   n_qubits); other values are SV_ERR_INVALID.  The results
 *                   are the same up to rounding; the choice changes the passes
 *                   and the kernel that runs them */
typedef enum { SV_BLOCK_AUTO = 0, SV_BLOCK_DENSE = 1 } sv_block_mode;
typedef struct sv_exec_opts {
  int32_t fuse_max_k;
  int32_t block_mode;
  int32_t ops_per_pass;
  int32_t tile_qubits;
} sv_exec_opts;

/* sv_apply_circuit with explicit options (opts NULL = all zero). */
sv_status sv_apply_circuit_ex(void* state, int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                              const double* param_values, size_t n_param_values, const sv_exec_opts* opts,
                              void* stream);

/* Expectation of each term, <psi|P_j|psi> (without c_j), evaluated by the
 * matrix-free Pauli action (Sec. 4.4), accumulated in double.
 *   state        device, not modified
 *   terms        host array of n_terms (1..4096)
 *   out          n_terms doubles: host memory when out_on_device == 0 (the
 *                call synchronizes `stream`), else device memory (the call
 *                only enqueues work)
 * Uses library-owned device scratch (allocated on first use per stream). */
sv_status sv_expect(const void* state, int n_qubits, sv_dtype dtype, const sv_pauli_term* terms, size_t n_terms,
                    double* out, int out_on_device, void* stream);

/* <Z_q> for every qubit q and their sum, in one read-only pass:
 * <Z_q> = sum_b |psi_b|^2 (-1)^{b_q} (Sec. 5.3 probabilities; Sec. 4.4).
 *   out  n_qubits + 1 doubles: out[q] = <Z_q>, out[n_qubits] = sum_q <Z_q>;
 *        host or device memory as selected by out_on_device (see sv_expect).
 * Uses library-owned device scratch (allocated on first use per stream). */
sv_status sv_expect_z_all(const void* state, int n_qubits, sv_dtype dtype, double* out, int out_on_device,
                          void* stream);

/* sv_expect_z_all without any device allocation.  (The paper has no
 * counterpart: this exists for callers that cannot let a library allocate
 * device memory -- a process whose device memory all belongs to its own pool
 * or allocator, or code that must not let a cudaMalloc/cudaFree synchronize
 * the device under other streams.)
 *   state  device, 2^n amplitudes of dtype, not modified
 *   out    device, n_qubits + 1 doubles, as sv_expect_z_all; the call only
 *          enqueues work on `stream`
 * The per-block partial sums live in a fixed array inside the library (1024
 * rows of 35 doubles, 280 KiB, held on every GPU that loads the library until
 * the process exits) instead of allocated scratch.  n_qubits outside 1..34, or
 * a GPU that would need more than 1024 partial rows, is SV_ERR_INVALID.  The
 * first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) and should come before any stream capture.  All calls
 * share the array: calls that overlap on the GPU race and may return wrong
 * values. */
sv_status sv_expect_z_all_noalloc(const void* state, int n_qubits, sv_dtype dtype, double* out, void* stream);

/* Planning summary of a circuit without running it (opts as in
 * sv_apply_circuit_ex, NULL = all zero): number of fused blocks (the paper's
 * fusion when 2 <= fuse_max_k <= 5, else the gate count), the number of
 * passes over the state the library would make, and, if
 * block_starts is not NULL, the index of the first gate of each block
 * (block_starts must hold n_gates + 1 ints; block_starts[blocks] = n_gates). */
sv_status sv_plan_info(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                       const double* param_values, size_t n_param_values, const sv_exec_opts* opts,
                       int* out_blocks, int* out_sweeps, int* block_starts);

/* Measurement probabilities (Sec. 5.3, measurement equation):
 * p_i = x_i^2 + y_i^2 for psi_i = x_i + i y_i, in double (each product and
 * the sum rounded once), divided by their sum when normalise != 0.
 *   state   device, 2^n amplitudes of `dtype`
 *   out     device, 2^n doubles (caller-owned)
 * Asynchronous on `stream`; errors as sv_expect. */
sv_status sv_probabilities(const void* state, int n_qubits, sv_dtype dtype, double* out, int normalise,
                           void* stream);

/* Finite-shot measurement (Sec. 5.3: basis indices drawn from the probability
 * vector), one draw per caller-supplied uniform u_k in [0, 1), by the inverse
 * of the cumulative distribution taken in exact integer arithmetic:
 *   q_i = floor(p_i 2^61) with p_i as in sv_probabilities (not normalised),
 *   Q = sum_i q_i,  t_k = floor(floor(u_k 2^53) Q / 2^53),
 *   index_k = the smallest i with q_0 + ... + q_i > t_k.
 * The result does not depend on any summation order, so the same uniforms
 * give the same indices on every device and on the host.
 *   uniforms  host, n_shots doubles in [0, 1) (else SV_ERR_INVALID)
 *   out       n_shots basis indices, host (out_on_device = 0: the call waits)
 *             or device memory
 * 5 <= n_qubits <= 34; a state with no mass above 2^-61 is SV_ERR_INVALID. */
sv_status sv_sample(const void* state, int n_qubits, sv_dtype dtype, const double* uniforms, size_t n_shots,
                    uint64_t* out, int out_on_device, void* stream);

/* Host execution of the pass kernel's programs: builds the plan of `gates`
 * exactly as sv_apply_circuit_ex would for `dtype` (fusion, tiles, register
 * phases, rotations, phase tables), then runs every program on the host in
 * double precision.  The paper has no counterpart: this validates the
 * program builder (the transformation of Sec. 5.3 / 9.2 gate lists into pass
 * programs) without a GPU, and says nothing about the kernel's arithmetic.
 *   state   host, 2^n complex128 (re, im interleaved), updated in place
 * 1 <= n_qubits <= 20; errors as sv_apply_circuit_ex.  Slow (seconds). */
sv_status sv_emulate_apply(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                           const double* param_values, size_t n_param_values, const sv_exec_opts* opts,
                           double* state);

/* Gradients of f_b(theta) = <0|U^dag(theta_b) H U(theta_b)|0> (Sec. 4.2) for a
 * batch of parameter vectors of one circuit template, by the adjoint method:
 * one forward pass storing the state every `checkpoint_every` gates, then
 * lambda = H psi (Sec. 4.4 matrix-free Pauli action) and one reverse pass that
 * un-applies the gates from psi and lambda and adds Im <lambda|G|psi> for
 * every rotation U = exp(-i theta G / 2) (equal to the parameter-shift
 * derivative of Sec. 4.2).  At each checkpoint the reverse pass replaces psi
 * by the stored forward state, which bounds the complex64 uncompute drift.
 *   gates            template; parameterised gates (param_slot[0] >= 0) must
 *                    be RX, RY, RZ, P, RXX, RYY, RZZ, EXC1 or EXC2 (else
 *                    SV_ERR_UNSUPPORTED); every gate has <= 2 targets except
 *                    double excitations (EXC2, 4 targets, at most 2
 *                    controls), which the adjoint runs as a controlled RY
 *                    between fixed CNOT/X permutations
 *   params           host, batch x n_params doubles, row-major; row b binds
 *                    the slots of state b
 *   terms            H = sum_j coeff_j P_j, 1..4096 terms
 *   checkpoint_every gates between stored states (0 = no checkpoints);
 *                    device memory grows by batch * 2^n amplitudes per stored
 *                    state
 *   out_grad         host, batch x n_params (slots no gate uses get 0; a slot
 *                    used by several gates gets the sum of their terms)
 *   out_value        host, batch values f_b
 * Library-owned device buffers (psi, lambda, checkpoints, tables) are kept
 * per stream and reused.  1 <= n_qubits <= 30, 1 <= batch <= 65535.
 * Synchronizes `stream`. */
sv_status sv_adjoint_grad(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates, const double* params,
                          int batch, int n_params, const sv_pauli_term* terms, size_t n_terms, int checkpoint_every,
                          double* out_grad, double* out_value, void* stream);

/* Checkpoint policy of the adjoint (Sec. 7.3: no checkpointing, a
 * user-selected interval, or automatic placement; discarded states are
 * recomputed in the backward pass).
 *   checkpoint_every     gates per segment: the reverse pass re-anchors psi
 *                        at every segment start (0 = never: psi is only
 *                        uncomputed, gate by gate)
 *   stored_states        -1: keep every segment-start state from the forward
 *                        pass (memory: segments x batch x 2^n amplitudes);
 *                        k >= 0: keep at most k of them, evenly spaced; the
 *                        others are recomputed in the reverse pass by applying
 *                        the gates again from the nearest kept state below
 *                        (or from |0..0>)
 *   memory_budget_bytes  > 0: automatic placement, stored_states = the number
 *                        of batch states the budget holds (overrides
 *                        stored_states) */
typedef struct sv_adjoint_opts {
  int32_t checkpoint_every;
  int32_t stored_states;
  double memory_budget_bytes;
} sv_adjoint_opts;

/* sv_adjoint_grad with a checkpoint policy (sv_adjoint_opts); the results are
 * the same whatever the policy, up to rounding. */
sv_status sv_adjoint_grad_ex(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                             const double* params, int batch, int n_params, const sv_pauli_term* terms,
                             size_t n_terms, const sv_adjoint_opts* opts, double* out_grad, double* out_value,
                             void* stream);

/* sv_adjoint_grad with a Hamiltonian per state: state b uses
 * H_b = sum_j row_coeffs[b * n_terms + j] P_j (the coeff field of `terms` is
 * not used).  This is the backward pass of a layer whose outputs are the
 * <P_j> of every state (Sec. 5.4 BatchLayer: per-qubit Z readout): with
 * row_coeffs = the upstream gradient dL/d<P_j>_b, out_grad is dL/dtheta.
 *   row_coeffs  host, batch x n_terms doubles
 * Every X-mask of the terms must fit one tile (13 qubits for complex64, 12 for
 * complex128, the lowest 5 / 4 included), else SV_ERR_UNSUPPORTED; Z-only
 * terms always do.  Other arguments and errors as sv_adjoint_grad. */
sv_status sv_adjoint_grad_rows(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                               const double* params, int batch, int n_params, const sv_pauli_term* terms,
                               size_t n_terms, const double* row_coeffs, int checkpoint_every, double* out_grad,
                               double* out_value, void* stream);

/* Forward pass of a batched circuit template (Sec. 4.1 BatchSV, Sec. 5.4
 * BatchLayer): state b = U(params_b)|0..0>, then <Z_q> for every qubit and
 * their sum, per state.  The template rules are those of sv_adjoint_grad
 * (parameterised gates are one-parameter rotations).
 *   out_z   host, batch x (n_qubits + 1) doubles: <Z_0> .. <Z_{n-1}>, sum
 * The call waits for the result.  1 <= n_qubits <= 30, 1 <= batch <= 65535. */
sv_status sv_batch_expect_z(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                            const double* params, int batch, int n_params, double* out_z, void* stream);

/* sv_adjoint_grad / sv_adjoint_grad_rows with every array in device memory:
 * the step of a training loop whose parameters, upstream gradients and
 * results stay on the GPU (Sec. 5.4 BatchLayer; Sec. 8.2 batched QML).  The
 * per-state gate matrices are built on the device from `params` (double
 * precision, narrowed once), so no parameter value crosses to the host; the
 * call only enqueues work on `stream` and returns.
 *   params      device, batch x n_params doubles (values are not checked on
 *               the host: a non-finite parameter gives non-finite results)
 *   row_coeffs  device, batch x n_terms doubles (H_b as in
 *               sv_adjoint_grad_rows, with its tile rule on X-masks), or NULL
 *               for H = sum_j terms[j].coeff P_j for every state
 *   out_grad    device, batch x n_params doubles, or NULL: values only (the
 *               forward pass and H psi, no reverse pass)
 *   out_value   device, batch doubles
 * Other arguments and errors as sv_adjoint_grad. */
sv_status sv_adjoint_grad_device(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                                 const double* params, int batch, int n_params, const sv_pauli_term* terms,
                                 size_t n_terms, const double* row_coeffs, int checkpoint_every, double* out_grad,
                                 double* out_value, void* stream);

/* sv_batch_expect_z with device arrays (params as sv_adjoint_grad_device;
 * out_z device, batch x (n_qubits + 1) doubles); only enqueues work. */
sv_status sv_batch_expect_z_device(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                                   const double* params, int batch, int n_params, double* out_z, void* stream);

/* ---- serving: packed small states -------------------------------------------
 * Runs many small independent circuits in ONE kernel launch: request b gets one
 * CTA that keeps its whole state (2^n amplitudes, n <= SV_SMALL_MAX_QUBITS) in
 * shared memory from |0..0> to the end, applies its gates (the same lowering,
 * fast paths and register phases as sv_apply_circuit) and writes
 * out_sum_z[b] = sum_q <Z_q>.  Small states never touch HBM; this packs the
 * launch-bound small requests of a serving stream (the paper's NPU runs of small
 * states were launch-bound, Sec. 9.3).
 *   n_qubits[b], gates[b], n_gates[b]  request b (host arrays, no slots)
 *   out_sum_z  n_requests doubles, host (call synchronizes) or device (async)
 * Library-owned pinned staging and device program buffers are kept per stream. */
#define SV_SMALL_MAX_QUBITS 12
sv_status sv_run_batch_small(int n_requests, sv_dtype dtype, const int* n_qubits, const sv_gate* const* gates,
                             const size_t* n_gates, double* out_sum_z, int out_on_device, void* stream);

/* ---- serving sessions: a resident packed kernel -------------------------------
 * A session keeps one kernel resident on `n_ctas` SMs (0: a sixteenth of the
 * SMs, at least 2) whose CTAs take small requests from a work queue while it
 * runs: the host publishes a request (its programs uploaded, its queue entry
 * written to pinned host memory mapped into the device), a free CTA claims it,
 * runs its circuit from |0..0> on a state held in shared memory (as
 * sv_run_batch_small does) and writes sum_q <Z_q> and a done word back to
 * mapped memory.  A request costs no kernel launch (Sec. 9.3: small states
 * were launch-bound on the NPU).  Requests up to SV_SESSION_MAX_QUBITS qubits
 * (complex64, whose sessions run 512-thread CTAs with 128 KiB of shared
 * memory for 14-qubit states; 12 qubits and 256 threads for complex128),
 * gates without parameter slots.
 * Every device-side wait is bounded: a CTA that finds no published request
 * for wait_limit_s seconds records SV_ERR_TIMEOUT and ends; the next submit
 * relaunches the kernel, and sv_small_session_stop reports the timeout.
 * A device-wide synchronization (cudaDeviceSynchronize, cudaFree,
 * cudaFreeHost ...) waits for the resident kernel, that is until its CTAs
 * have found no work for wait_limit_s: keep the limit short (tens of
 * milliseconds) where such calls can happen while a session is live.
 * While a session is live, the TMA pass of apply calls on the same device
 * runs on the SMs the session's CTAs leave free, and loading a compiled pass
 * kernel pauses the session around the load (sv_jit_set_mode).  A session
 * belongs to the device current at start; its calls are thread-safe. */
#define SV_SESSION_MAX_QUBITS 14
typedef struct sv_small_session sv_small_session;
/* capacity: requests in flight at most (1..2^20); arena_programs: pass
 * programs held for them (1..65536, about 32 KB each on the device). */
sv_status sv_small_session_start(sv_dtype dtype, int capacity, int arena_programs, double wait_limit_s, int n_ctas,
                                 sv_small_session** out);
/* Plans and publishes n_requests requests (host arrays as sv_run_batch_small);
 * tickets[b] identifies request b.  SV_ERR_OOM when the session holds
 * `capacity` requests in flight or its program arena is full: poll, then
 * submit again. */
sv_status sv_small_session_submit(sv_small_session* s, int n_requests, const int* n_qubits,
                                  const sv_gate* const* gates, const size_t* n_gates, int64_t* tickets);
/* *done = 1 and *result = sum_q <Z_q> once the ticket is done, else *done = 0
 * (never waits).  A ticket older than `capacity` later ones is SV_ERR_INVALID. */
sv_status sv_small_session_poll(sv_small_session* s, int64_t ticket, double* result, int* done);
/* Asks the kernel to end once no published request is left, waits for it and
 * frees the session.  SV_ERR_TIMEOUT if any of its waits ran out (the session
 * sat idle past its limit, or was never given work); results of done
 * tickets are valid either way. */
sv_status sv_small_session_stop(sv_small_session* s);

/* End-to-end call on HOST buffers: copies `state_in` (host, 2^n amplitudes of
 * dtype; NULL means |0..0>) to a library-owned device buffer, applies the
 * circuit as sv_apply_circuit does, evaluates <Z_q> for all qubits into
 * out_z (host, n_qubits + 1 doubles, as sv_expect_z_all) and, when
 * state_out is not NULL, copies the final state back to it (host).  The
 * device buffer is kept per stream and reused by later calls of the same
 * or smaller size.  Synchronizes `stream`.
 * Host state buffers (here and in sv_set_state / sv_get_state) must hold
 * 2^n amplitudes of dtype.  When one is page-locked memory mapped into the
 * device at the same address (cudaHostAlloc / cudaMallocHost, pinned torch
 * tensors) and 16-byte aligned, the copy runs as a kernel of SM loads and
 * stores over the CPU-GPU link (launched on `stream`, family "host_load" /
 * "host_store" in the kernel timing below); on GB300 this keeps its rate when
 * the link has been idle, where a copy-engine transfer started behind the
 * circuit's kernels was measured several times slower.  Any other host
 * memory is copied with cudaMemcpyAsync. */
sv_status sv_run_host(int n_qubits, sv_dtype dtype, const void* state_in, const sv_gate* gates, size_t n_gates,
                      const double* param_values, size_t n_param_values, int fuse_max_k, double* out_z,
                      void* state_out, void* stream);

/* ---- library-owned states ------------------------------------------------
 * For callers without their own device allocator.  A handle owns one device
 * buffer of 2^n amplitudes of dtype, bound to `stream` (Sec. 4.1: the dense
 * State; Sec. 5.1: conversion to the host is an explicit exit). */
typedef struct sv_state* sv_handle;

/* Allocates a state initialised to |0..0>.  SV_ERR_OOM if cudaMalloc fails. */
sv_status sv_alloc(int n_qubits, sv_dtype dtype, void* stream, sv_handle* out);
/* Frees the state (after synchronizing its stream).  NULL is a no-op. */
sv_status sv_free(sv_handle h);
/* Device pointer of the state's amplitudes (for the pointer-based calls). */
void* sv_state_ptr(sv_handle h);
/* Copies 2^n amplitudes of the handle's dtype from `src` (host memory when
 * src_is_device == 0, else device memory) into the state.  Synchronizes. */
sv_status sv_set_state(sv_handle h, const void* src, int src_is_device);
/* Copies the state into `dst` (host or device as selected).  Synchronizes. */
sv_status sv_get_state(sv_handle h, void* dst, int dst_is_device);

/* ---- kernel timing ---------------------------------------------------------
 * When enabled, the library brackets each of its kernel launches with a pair
 * of CUDA events recorded on the launching stream, so the per-launch device
 * time is measured where the work runs (median-free totals; the caller times
 * whole steps itself).  Entries aggregate by kernel family. */
typedef struct sv_profile_entry {
  char name[32];       /* kernel family, e.g. "sweep", "expect_z_all" */
  int64_t launches;
  double total_ms;     /* sum of event-measured launch durations */
  double bytes;        /* sum of algorithmic HBM bytes of those launches */
} sv_profile_entry;

/* on != 0 starts recording (clearing earlier records); 0 stops. */
sv_status sv_profile_enable(int on);
/* Waits for the recorded events and writes up to max_entries aggregates;
 * *n_out = number of families.  reset != 0 clears the records. */
sv_status sv_profile_read(sv_profile_entry* out, int max_entries, int* n_out, int reset);

/* Releases the library's device scratch buffers of every stream (after a
 * device synchronize).  Later calls allocate them again. */
sv_status sv_release_scratch(void);

/* ---- pass kernels compiled at run time -------------------------------------
 * A pass over a large complex64 state (the tiled gate application of Sec. 5.3
 * with the gates of one pass applied per tile) normally runs a kernel that
 * interprets the pass program.  The library can instead write each program
 * out as straight-line CUDA (every op's kind, register slots, controls and
 * coefficient offsets as constants), compile it with NVRTC for the current
 * device and launch that kernel in its place: same tile movement, same
 * arithmetic in the same order (bit-identical results), fewer instructions.
 * Kernels are kept by program structure (the gates and their qubits, not their
 * angles), so every circuit of the same structure -- a variational template at
 * new parameters, the requests of one serving family -- shares them.
 * Compilation runs on host threads (about a second per distinct program, at
 * most one per host core across the process) and its kernels are cached for
 * the life of the process, per device.  Loading a compiled module waits for
 * every resident kernel of the device, so live serving sessions on the device
 * are paused for the load (their kernels end and relaunch; requests in flight
 * are kept).  On states with fewer than 2^21 amplitudes, for complex128 states
 * and where NVRTC is missing, the interpreting kernels run.
 *
 * mode: 0 never compile; 1 (default) compile a program structure on its second
 * use (by any circuit); 2 on its first; -1 take the SV_JIT environment variable
 * (0, 1, 2).  Other values are SV_ERR_INVALID. */
sv_status sv_jit_set_mode(int mode);
/* Current mode, whether NVRTC was found (available), kernels compiled and
 * failed so far, launches of compiled kernels, host seconds spent compiling;
 * message (host, message_cap bytes, NUL-terminated) gets why NVRTC is missing,
 * else the last compile error (empty if none).  Any pointer may be NULL. */
sv_status sv_jit_info(int* mode, int* available, long long* compiled, long long* failed, long long* launches,
                      double* compile_seconds, char* message, size_t message_cap);
/* Plans a circuit as sv_apply_circuit_ex would and generates the kernel source
 * of every pass that would run compiled (*n_sources); with compile != 0 also
 * compiles each for sm_<arch>a (arch e.g. 103) and counts successes in
 * *n_compiled.  Needs no device.  text (host, text_cap bytes, NUL-terminated,
 * truncated to fit) receives the first compile error, else every source, each
 * followed by a line "// ----".  SV_ERR_UNSUPPORTED if compile
 * is asked for and NVRTC is missing. */
sv_status sv_jit_check(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates, const double* param_values,
                       size_t n_param_values, const sv_exec_opts* opts, int compile, int arch, int* n_sources,
                       int* n_compiled, char* text, size_t text_cap);
/* The adjoint's batched passes (sv_adjoint_grad and the calls that share its
 * sweeps) are compiled the same way, per circuit template: a template's calls
 * are counted by its structure (gates without their angles, checkpoint
 * interval and state size), and on the call the mode names every
 * batched program of the call is compiled and its kernel launched in place
 * of the interpreting one (bit-identical gradients and values).
 * sv_jit_check_adjoint writes (and with compile != 0 compiles for sm_<arch>a)
 * the distinct kernels of a template's forward and reverse passes without a
 * device, as sv_jit_check; n_params bounds the gates' parameter slots. */
sv_status sv_jit_check_adjoint(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates, int n_params,
                               int checkpoint_every, int compile, int arch, int* n_sources, int* n_compiled,
                               char* text, size_t text_cap);

#ifdef __cplusplus
}
#endif

#endif /* SV_H */
