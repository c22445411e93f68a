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
#include "sv_pass_ops.cuh"
#include "sv_tma_pass.cuh"

namespace sv {

namespace {


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
      r_phase_table<R, RQ>(v, T0);
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


// ---------------------------------------------------------------- kernels

// Runs every phase of a program on a tile that is already in shared memory.
// KMAX: widest dense operation the program runs in shared memory; RQ: the
// register qubits of its register phases.
struct NoRelease {
  __device__ __forceinline__ void operator()() const {}
};


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
    stage_copy_out<R>(s, tsz, gstate, base, h, gr);
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
// accelerator: one CTA per SM, NC groups of 128 threads, a ring of
// mbarrier-guarded shared-memory stages filled by 5-D tensor copies, the last
// register phase storing straight to the state (sv_tma_pass.cuh).  Here the
// groups interpret the program; sv_jit.cpp compiles straight-line runners of
// single programs into the same scaffold.  A wait that runs out records
// SV_ERR_TIMEOUT in g_sweep_status.

__device__ int g_sweep_status = 0;  // SV_OK, or the first error a pass kernel recorded
static_assert(kTmaStatusTimeout == (int)SV_ERR_TIMEOUT, "pass kernel timeout status");

// Threads of a group: 2^(m - RQ), 128 for 12-qubit tiles with five register
// qubits (32 amplitudes a thread).  Sixteen amplitudes a thread (256-thread
// groups, 24 warps an SM at 80 registers) measured slower: 7.55 against 5.65
// ms per 30-qubit pass, the per-phase work of a thread spread over half the
// amplitudes and a third more phases.
template <int RQ>
constexpr int tma_group_threads() {
  return RQ == 5 ? 128 : 256;
}

// Runs a program's phases on one tile by interpreting them.
template <typename R, int KMAX, int RQ, int OPS>
struct InterpRunner {
  const SweepProgram<R>& P;
  template <class Release>
  __device__ __forceinline__ void operator()(Cx<R>* s, const Cx<R>* coef, uint64_t base, const Grp& gr,
                                             Cx<R>* state, const Release& release) const {
    run_phases<R, KMAX, RQ, OPS, true>(P, coef, s, 1 << P.h.m, base, gr, state, release);
  }
};

template <typename R, int KMAX, int RQ, int OPS, int NC>
__global__ void __launch_bounds__(NC * tma_group_threads<RQ>(), 1)
    k_sweep_tma(Cx<R>* __restrict__ state, const __grid_constant__ CUtensorMap tmap,
                const __grid_constant__ TmaBoxes bx, const __grid_constant__ SweepProgram<R> P, int ns) {
  tma_pass_body<R, NC, tma_group_threads<RQ>()>(state, &tmap, bx, P.h, P.coef, ns, &g_sweep_status,
                                                InterpRunner<R, KMAX, RQ, OPS>{P});
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
  // the sum runs over the first kRedThreads threads in a fixed order, so a
  // request's result does not depend on the CTA's size (the packed launch and
  // both session kernels give the same bits)
  constexpr int kRedThreads = 256;
  double acc = 0.0;
  if (threadIdx.x < kRedThreads)
    for (int a = threadIdx.x; a < tsz; a += kRedThreads) {
      const Cx<R> x = s[phys<R>(a)];
      acc += (double)(x.re * x.re + x.im * x.im) * (double)(n - 2 * __popc(a));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && threadIdx.x < kRedThreads) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kRedThreads / 32; w++) t += red[w];
    result = t;
  }
}

// NT threads a CTA: 256 (a register group of 16 or 32 amplitudes per thread
// covers states up to 13 qubits), or 512 for sessions that take 14-qubit
// complex64 requests (2^9 groups of 32; 128 KiB of shared memory).
template <typename R, int NT>
__global__ void __launch_bounds__(NT) k_small_session(SmallSessionDev d, const SweepProgram<R>* __restrict__ progs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<R>* s = reinterpret_cast<Cx<R>*>(smem_raw);
  __shared__ double red[NT / 32];
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
  return (size_t)tma_smem_bytes_of<R>(h.m, h.ncoef, ns);
}

// Stages of a TMA pass: as many as shared memory holds (more than the groups).
template <typename R>
static int tma_stages(const ProgramHeader& h) {
  int ns = kTmaMaxStages;
  while (ns > kTmaGroups && tma_smem_bytes<R>(h, ns) > 227 * 1024) ns--;
  return ns > kTmaGroups ? ns : 0;
}

// Device address of g_sweep_status (per device), for compiled pass kernels.
static int* sweep_status_ptr() {
  static int* ptr[64] = {nullptr};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sweep_status) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptr[dev] = (int*)p;
  }
  return ptr[dev];
}

static uint64_t tma_grid(uint64_t ntiles);

template <typename R, int KMAX, int RQ, int OPS>
static cudaError_t launch_sweep_tma_k(Cx<R>* state, const SweepProgram<R>& prog, const CUtensorMap& map,
                                      const TmaBoxes& bx, cudaStream_t stream) {
  constexpr int NC = kTmaGroups;
  const int ns = tma_stages<R>(prog.h);
  if (ns == 0) return cudaErrorInvalidConfiguration;
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
  const uint64_t grid = tma_grid(1ull << (prog.h.n - prog.h.m));
  k_sweep_tma<R, KMAX, RQ, OPS, NC>
      <<<(unsigned)grid, NC * tma_group_threads<RQ>(), smem, stream>>>(state, map, bx, prog, ns);
  return cudaGetLastError();
}

// Whether the TMA pass runs this program: complex64 states of at least 2^9
// tiles whose tile groups are 128 threads (12-qubit tiles with five register
// qubits), unless SV_SWEEP_TMA=0 in the environment selects the cp.async
// kernel.  (complex128 passes are bound by the FP64 pipe, and at the 128
// registers of four 128-thread groups per SM their register phases spill.)
static std::atomic<int> g_live_sessions[64];
static std::atomic<int> g_session_ctas[64];

void session_opened(int device, int ctas) {
  if (device < 0 || device >= 64) return;
  g_live_sessions[device]++;
  g_session_ctas[device] += ctas;
}
void session_closed(int device, int ctas) {
  if (device < 0 || device >= 64) return;
  g_live_sessions[device]--;
  g_session_ctas[device] -= ctas;
}
bool session_live(int device) { return device >= 0 && device < 64 && g_live_sessions[device].load() > 0; }

static bool tma_enabled() {
  const char* e = std::getenv("SV_SWEEP_TMA");
  return !(e && e[0] == '0');
}

// CTAs of a TMA pass (one per SM, each with a fixed share of the tiles): the
// SMs, less one per resident CTA of the device's live serving sessions (their
// shared memory leaves no room for a TMA CTA beside them), so that every CTA
// of the pass can be resident at once; at most one per tile.
static uint64_t tma_grid(uint64_t ntiles) {
  int dev = 0;
  cudaGetDevice(&dev);
  int64_t sms = device_sm_count();
  if (dev >= 0 && dev < 64) sms -= g_session_ctas[dev].load();
  const uint64_t g = sms < 1 ? 1 : (uint64_t)sms;
  return g < ntiles ? g : ntiles;
}

template <typename R, int RQ>
static cudaError_t launch_sweep_tma(Cx<R>* state, const SweepProgram<R>& prog, cudaStream_t stream, bool& used,
                                    const JitKernel* jit, bool& used_jit) {
  used = used_jit = false;
  if (!tma_enabled() || prog.h.n - prog.h.m < 9 || (1 << (prog.h.m - RQ)) != tma_group_threads<RQ>())
    return cudaSuccess;
  CUtensorMap map;
  TmaBoxes bx;
  if (!tma_map_for<R>(state, prog.h, map, bx)) return cudaSuccess;
  if (jit) {  // the program's own compiled kernel, same arguments and launch shape
    const int ns = tma_stages<R>(prog.h);
    int* status = sweep_status_ptr();
    if (ns && status) {
      const uint64_t grid = tma_grid(1ull << (prog.h.n - prog.h.m));
      used = used_jit = true;
      return jit_launch(jit, state, &map, &bx, &prog, ns, status, (unsigned)grid,
                        kTmaGroups * tma_group_threads<RQ>(), tma_smem_bytes<R>(prog.h, ns), stream);
    }
  }
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
cudaError_t launch_sweep(Cx<R>* state, const SweepProgram<R>& prog, cudaStream_t stream, const char** kernel,
                         const JitKernel* jit) {
  // four register qubits with two tile buffers, or five with one (12-qubit
  // complex64 tiles; complex128 tiles have 11 qubits); large complex64 states
  // take the TMA pass, with the program's compiled kernel when it has one
  bool used = false, used_jit = false;
  if (kernel) *kernel = "sweep";
  if constexpr (sizeof(R) == 4) {
    if (prog.h.rq == 5) {
      cudaError_t e = launch_sweep_tma<R, 5>(state, prog, stream, used, jit, used_jit);
      if (used && kernel) *kernel = used_jit ? "sweep_jit" : "sweep_tma";
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

template <typename R, int NT>
cudaError_t launch_small_session_nt(const SmallSessionDev& d, const SweepProgram<R>* progs, int smem, int grid,
                                    cudaStream_t stream) {
  static int configured_bytes[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem > 48 * 1024 && smem > configured_bytes[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_small_session<R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured_bytes[dev] = smem;
  }
  k_small_session<R, NT><<<grid, NT, smem, stream>>>(d, progs);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_small_session(const SmallSessionDev& d, const SweepProgram<R>* progs, int max_n, int grid,
                                 cudaStream_t stream) {
  const int smem = (int)sizeof(Cx<R>) << max_n;
  if constexpr (sizeof(R) == 4)
    if (max_n >= 14) return launch_small_session_nt<R, 512>(d, progs, smem, grid, stream);
  return launch_small_session_nt<R, 256>(d, progs, smem, grid, stream);
}

template cudaError_t launch_small_session<float>(const SmallSessionDev&, const SweepProgram<float>*, int, int,
                                                 cudaStream_t);
template cudaError_t launch_small_session<double>(const SmallSessionDev&, const SweepProgram<double>*, int, int,
                                                  cudaStream_t);
template cudaError_t launch_small_batch<float>(const SweepProgram<float>*, const int*, const int*, int, int, double*,
                                               cudaStream_t);
template cudaError_t launch_small_batch<double>(const SweepProgram<double>*, const int*, const int*, int, int, double*,
                                                cudaStream_t);
template cudaError_t launch_sweep<float>(Cx<float>*, const SweepProgram<float>&, cudaStream_t, const char**,
                                         const JitKernel*);
template cudaError_t launch_sweep<double>(Cx<double>*, const SweepProgram<double>&, cudaStream_t, const char**,
                                          const JitKernel*);
template cudaError_t launch_init_basis<float>(Cx<float>*, int, uint64_t, cudaStream_t);
template cudaError_t launch_init_basis<double>(Cx<double>*, int, uint64_t, cudaStream_t);

}  // namespace sv
