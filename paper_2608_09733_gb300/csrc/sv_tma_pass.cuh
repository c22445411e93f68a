// sv_tma_pass.cuh -- the TMA pass over a state, shared by the library's pass
// kernel (sv_sweep.cu, which runs the pass program by interpreting it) and the
// kernels compiled at run time from one pass program (sv_jit.cpp, straight-line
// code).  Device code only, with no host headers, so the run-time compiler
// takes it as it is.
//
// One CTA per SM walks its tiles (tile = blockIdx.x + k * gridDim.x) through a
// ring of `ns` shared-memory stages (tile k in stage k mod ns):
//   - a tile is 16 boxes of 2 KiB, each box the 2^(E+4) amplitudes of local
//     bits 0..E+3, where 2^E amplitudes make one 128-byte row (E = 4 for
//     complex64, 3 for complex128).  A five-dimensional tensor map per pass
//     describes the state as [2^(n-q3)][2^(q3-q2)][2^(q2-q1)][2^(q1-E)][row],
//     q1..q3 being the tile qubits at local positions E+1..E+3; a box takes two
//     entries of each outer dimension.  The 128-byte swizzle of the copies
//     places amplitude l at phys(l), the XOR layout the register phases read;
//   - NC groups of T threads each take every NC-th tile: wait for its stage to
//     fill, run the pass program on it (a named barrier per group).  The
//     runner's last register phase loads its registers, meets the group's
//     barrier and calls release() -- warp 0 of the group then refills the
//     stage with the tile ns places further on -- and stores its results
//     straight to the state.  A lane of the loading warp issues one box each.
// So ns - NC tiles are loading while the groups compute, and no compute
// thread spends instructions on tile copies.  There is no separate producer
// warp: a 17th warp would cap the compute threads' registers at 96 (the
// register file is split between the SM's four schedulers).
//
// Every wait is bounded (one second of %globaltimer): a wait that runs out
// records the timeout status in *status, the CTA's groups stop waiting (they
// carry on over whatever the stages hold, so every thread keeps meeting its
// group's barriers), and the loads already issued are waited for (bounded)
// before the CTA exits.
#pragma once

#include "sv_pass_ops.cuh"

namespace sv {

constexpr int kTmaStatusTimeout = 5;  // SV_ERR_TIMEOUT
constexpr int kTmaBoxBytes = 2048;
constexpr int kTmaMaxStages = 8;
static_assert(kTmaMaxStages * 8 % 16 == 0 && 2 * kTmaMaxStages + 1 <= 20, "TMA pass shared-memory layout");
constexpr unsigned long long kTmaWaitLimitNs = 1000000000ull;

// Box geometry of a pass, passed beside its tensor map: the tile qubits at
// local positions E+1..E+3 (q1..q3) and above E+3 (hq[], the box index bits).
struct TmaBoxes {
  int q1, q2, q3;
  int nhq;
  int hq[kMaxTileQ];
};

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
// kTmaWaitLimitNs.  Gives up early when another thread of the CTA has already
// given up (*cta_flag != 0; pass NULL to wait regardless).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, volatile int* cta_flag, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; it++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 15u) == 0) {
      if (cta_flag && *cta_flag) return false;
      if (global_ns() - t0 > kTmaWaitLimitNs) {
        atomicCAS(status, 0, kTmaStatusTimeout);
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
// Waits until *tag == want (read with acquire), for at most kTmaWaitLimitNs
// (give-up rules as mbar_wait_bounded).
__device__ __forceinline__ bool tag_wait_bounded(const volatile uint32_t* tag, uint32_t want, volatile int* cta_flag,
                                                 int* status) {
  if (ld_acquire_u32(tag) == want) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; it++) {
    if (ld_acquire_u32(tag) == want) return true;
    if ((it & 15u) == 0) {
      if (*cta_flag) return false;
      if (global_ns() - t0 > kTmaWaitLimitNs) {
        atomicCAS(status, 0, kTmaStatusTimeout);
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

template <typename R>
__device__ __forceinline__ void tma_coords(uint64_t g, const TmaBoxes& bx, int& c1, int& c2, int& c3, int& c4) {
  constexpr int E = sizeof(Cx<R>) == 8 ? 4 : 3;
  c1 = (int)((g >> E) & ((1ull << (bx.q1 - E)) - 1ull));
  c2 = (int)((g >> bx.q1) & ((1ull << (bx.q2 - bx.q1)) - 1ull));
  c3 = (int)((g >> bx.q2) & ((1ull << (bx.q3 - bx.q2)) - 1ull));
  c4 = (int)(g >> bx.q3);
}

// Shared memory of a TMA pass with ns stages of 2^m amplitudes and a pool of
// ncoef coefficients.
template <typename R>
__host__ __device__ constexpr unsigned long long tma_smem_bytes_of(int m, int ncoef, int ns) {
  return 1024ull + (unsigned long long)ns * ((unsigned long long)sizeof(Cx<R>) << m) +
         (unsigned long long)sizeof(Cx<R>) * (unsigned long long)((ncoef + 1) & ~1) + 16ull * kTmaMaxStages + 16ull +
         32ull + 16ull * 32ull;
}

// The body of a TMA pass kernel (see the top of this file).  runner(stage,
// coef, base, grp, state, release) runs the pass program on one tile: `stage`
// holds it in shared memory, `coef` is the coefficient pool copied to shared
// memory, `base` the tile's global base index; the runner calls release()
// after its last phase's registers are loaded and stores the tile to `state`.
template <typename R, int NC, int T, class Runner>
__device__ __forceinline__ void tma_pass_body(Cx<R>* __restrict__ state, const void* tmap, const TmaBoxes& bx,
                                              const ProgramHeader& h, const Cx<R>* coef_src, int ns, int* status,
                                              const Runner& runner) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t tile_bytes = (uint32_t)sizeof(Cx<R>) << h.m;
  // stages from the first 1024-byte boundary (the swizzle pattern's period),
  // then the coefficient pool, the stage barriers, the loads issued into each
  // stage, the stages' tile tags, the CTA's give-up flag, per-CTA constants
  // and the coordinate offsets of each box of a tile
  const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
  unsigned char* stages = smem_raw + pad;
  Cx<R>* scoef = reinterpret_cast<Cx<R>*>(stages + (size_t)ns * tile_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(scoef + ((h.ncoef + 1) & ~1));
  unsigned* issued = reinterpret_cast<unsigned*>(bars + kTmaMaxStages);
  volatile uint32_t* stage_tile = reinterpret_cast<volatile uint32_t*>(issued + kTmaMaxStages);
  volatile int* flag = reinterpret_cast<volatile int*>(stage_tile + kTmaMaxStages);
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
      tma_load5(st0 + b * tile_bytes + lane * kTmaBoxBytes, tmap, c1 + bc.x, c2 + bc.y, c3 + bc.z, c4 + bc.w,
                full0 + 8 * b);
    }
  };
  for (int c = threadIdx.x; c < h.ncoef; c += blockDim.x) scoef[c] = coef_src[c];
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
  const Grp gr{threadIdx.x % T, (uint32_t)T, 1u + g};
  const bool loader = gr.tid < 32;  // warp 0 of the group refills the stages it frees
  uint64_t base = tile_base(g);
  for (uint64_t k = g; k < K; k += NC, base = dep_add(base, cst[1])) {
    const uint32_t b = (uint32_t)(k % (uint64_t)ns);
    // a wait that runs out sets the CTA's flag and the group carries on over
    // whatever the stage holds: every thread keeps meeting the group's
    // barriers, so nothing waits forever, and the status says the pass failed
    if (tag_wait_bounded(stage_tile + b, (uint32_t)k, flag, status))
      mbar_wait_bounded(full0 + 8 * b, (uint32_t)((k / ns) & 1), flag, status);
    auto release = [&]() {
      if (loader && k + ns < K && __all_sync(0xffffffffu, *flag == 0)) load_tile(b, k + ns, dep_add(base, cst[2]));
    };
    runner(reinterpret_cast<Cx<R>*>(stages + (size_t)b * tile_bytes), scoef, base, gr, state, release);
  }
  __syncthreads();
  if (threadIdx.x == 0 && *flag)  // stopped early: loads still in flight must land first
    for (int b = 0; b < ns; b++)
      if (issued[b]) mbar_wait_bounded(full0 + 8 * b, (issued[b] - 1) & 1u, nullptr, status);
}

}  // namespace sv
