// sv_jit.cpp -- pass kernels compiled at run time from one program.
//
// The library's pass kernel interprets a program: for every op of every
// register phase it loads the op's dispatch word, branches on its kind and
// slots, and computes its conditions and table variants, once per tile per
// thread.  On large states that bookkeeping costs as many issue slots as the
// arithmetic.  Here a program is written out as straight-line CUDA -- every
// phase's register positions, every op's kind, slots, controls, coefficient
// offsets and sign patterns as constants -- calling the same register and
// shared-memory op functions (sv_pass_ops.cuh) inside the same TMA pass
// scaffold (sv_tma_pass.cuh), compiled with NVRTC for the device's
// architecture and launched in place of the interpreting kernel.  The
// arithmetic is the same sequence of operations, so both kernels give the
// same bits.
//
// The adjoint's batched programs are compiled the same way
// (jit_batch_source: every phase and op as a constant, direct calls to the
// register-op functions of sv_batch_ops.cuh inside its tile loop).
//
// NVRTC is opened with dlopen on first use; without it (or the driver's
// module entry points) every pass keeps the interpreting kernel.  A compiled
// kernel is cached per (device, source text) for the life of the process and
// found by program structure (jit_program_kernels) or batched program
// (jit_batch_lookup).  Compiles run on host threads, at most one per host core
// across the process; a module load pauses the device's serving sessions
// (a load waits for every resident kernel to end).
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sv_adjoint.h"
#include "sv_internal.h"
#include "sv_jit_headers.inc"  // kJitHeaderNames / kJitHeaderTexts, written by build.py

namespace sv {

struct JitKernel {
  CUfunction fn = nullptr;
  int device = -1;
  std::atomic<size_t> smem_configured{0};  // dynamic shared memory the function allows
};

namespace {

// ---------------------------------------------------------------- source

struct Src {
  std::string s;
  void line(const char* fmt, ...) __attribute__((format(printf, 2, 3))) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    const int n = vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (n >= (int)sizeof(buf)) {  // a longer line: format it again at its length
      std::string big((size_t)n + 1, '\0');
      va_start(ap, fmt);
      vsnprintf(&big[0], big.size(), fmt, ap);
      va_end(ap);
      big.resize((size_t)n);
      s += big;
    } else if (n > 0) {
      s += buf;
    }
    s += '\n';
  }
};

// Groups of a CTA and their threads, as the interpreting TMA pass: four
// groups of 128 threads (12-qubit tiles, five register qubits).  Measured on
// the 30-qubit layered circuit: three groups 3.73 ms a pass, four 3.59.
constexpr int kJitGroups = 4;
constexpr int kJitGroupThreads = 128;

// 128-byte lines that warp 0's stores touch, summed over its store
// instructions, when the last register phase `ph` writes its registers
// straight to the state (16-byte pairs with local bit 0 in slot 0, else
// 8-byte stores).  A coalesced store of 32 lanes touches 4 lines (16-byte) or
// 2 (8-byte): 64 in all.  When the phase holds the tile's low local bits in
// registers, the lanes differ only in high bits and every store instruction
// lands in up to 32 lines, each written in part: the L1 data pipe, which also
// carries the register phases' shared-memory traffic, then takes 8x the
// wavefronts (measured: 1.4 ms against 0.66 ms for a 28-qubit pass of the
// same traffic).
int direct_store_lines(const ProgramHeader& h, const Phase& ph, int rq) {
  const bool pairs = ph.rp[0] == 0;
  int lines = 0;
  for (int j = 0; j < (1 << rq); j += pairs ? 2 : 1) {
    uint64_t seen[32];
    int ns = 0;
    for (uint32_t lane = 0; lane < 32; lane++) {
      uint32_t l = lane;
      for (int i = 0; i < rq; i++) {
        const uint32_t lo = l & ((1u << ph.rp[i]) - 1u);
        l = ((l >> ph.rp[i]) << (ph.rp[i] + 1)) | lo;
      }
      for (int i = 0; i < rq; i++)
        if ((j >> i) & 1) l |= 1u << ph.rp[i];
      uint64_t g = 0;
      for (int b = 0; b < h.m; b++)
        if ((l >> b) & 1u) g |= 1ull << h.tq[b];
      const uint64_t line = (g * 8ull) >> 7;
      bool dup = false;
      for (int t = 0; t < ns && !dup; t++) dup = seen[t] == line;
      if (!dup) seen[ns++] = line;
    }
    lines += ns;
  }
  return lines;
}
// The last register phase stores through shared memory and a coalesced copy
// when its direct stores would touch more lines than this a warp: the copy
// costs a warp 64 wavefronts to store the phase in shared memory, 64 to load
// it back and 64 lines of stores, 192 in all.
constexpr int kDirectStoreMaxLines = 192;

// ---------------------------------------------------------------- layouts
//
// Where a tile sits in shared memory between two phases.  Local amplitude l
// is at slot l ^ (XOR of col[b - 4] over the set bits b >= 4 of l), every col
// a value in slot bits 1..3: slot bit 0 is l's own, so 16-byte pairs stay
// whole and in order, and bits 1..3 change by a function of bits 4..11 only,
// so the map is one to one.  The TMA copies leave a stage in the 128-byte
// swizzle (phys()): bits 4, 5, 6 into slot bits 1, 2, 3.  Between two
// register phases (and before the copy-out) the layout is free, and the one
// picked lets both the phase that stores the tile and the one that loads it
// reach every bank: with phys() alone, a phase holding local bits 1..4 in
// registers and 16-byte pairs (or one whose lanes cannot spread over the
// 8-byte banks) takes its accesses in two or four times the wavefronts.
struct Layout {
  uint32_t col[8];
};
constexpr Layout kPhysLayout = {{2u, 4u, 8u, 0u, 0u, 0u, 0u, 0u}};

uint32_t slot_of(const Layout& L, uint32_t l) {
  uint32_t s = l;
  for (int b = 4; b < 12; b++)
    if ((l >> b) & 1u) s ^= L.col[b - 4];
  return s;
}

// The local bits a register phase's lanes hold: the thread's bits (the tile
// bits not in registers, ascending, as ins0 deposits them), the lowest five.
void lane_bits(const uint8_t* rp, int rq, int (&lb)[5]) {
  int n = 0;
  for (int b = 0; b < 12 && n < 5; b++) {
    bool reg = false;
    for (int i = 0; i < rq; i++) reg = reg || rp[i] == b;
    if (!reg) lb[n++] = b;
  }
}

// How many times the conflict-free count of wavefronts one warp access takes
// through L.  16-byte pairs go a quarter-warp at a time (lanes 0..7 should
// reach the 8 granules of a 128-byte row); 8-byte amplitudes a half-warp at
// a time (lanes 0..15 over 16 eight-byte banks).  The lanes' other bits add
// the same XOR to every slot, so they do not matter.
int access_ways(const Layout& L, const int (&lb)[5], bool pairs) {
  const int g = pairs ? 3 : 4;
  int count[16] = {0};
  int worst = 0;
  for (int x = 0; x < (1 << g); x++) {
    uint32_t l = 0;
    for (int i = 0; i < g; i++)
      if ((x >> i) & 1) l |= 1u << lb[i];
    const uint32_t sl = slot_of(L, l);
    const uint32_t key = pairs ? (sl >> 1) & 7u : sl & 15u;
    worst = std::max(worst, ++count[key]);
  }
  return worst;
}

// The layout of the boundary after register phase `st`, loaded next by
// register phase `ld` or (ld == nullptr) by the copy-out, whose lanes take
// local bits 1..5 in 16-byte pairs.  Candidates come in a fixed order, phys()
// first, so a program always gets the same source: the first whose accesses
// on both sides are conflict-free, else the best seen.
Layout choose_layout(const Phase& st, const Phase* ld, int rq) {
  int lst[5], lld[5];
  lane_bits(st.rp, rq, lst);
  const bool pst = st.rp[0] == 0;
  bool pld = true;
  if (ld) {
    lane_bits(ld->rp, rq, lld);
    pld = ld->rp[0] == 0;
  } else {
    for (int i = 0; i < 5; i++) lld[i] = i + 1;
  }
  auto cost = [&](const Layout& L) { return access_ways(L, lst, pst) + access_ways(L, lld, pld); };
  Layout best = kPhysLayout;
  int bc = cost(best);
  uint32_t x = 0x9E3779B9u;
  for (int t = 0; t < 20000 && bc > 2; t++) {
    Layout L;
    for (int b = 0; b < 8; b++) {
      x ^= x << 13;
      x ^= x >> 17;
      x ^= x << 5;
      L.col[b] = ((x >> 7) & 7u) << 1;
    }
    const int c = cost(L);
    if (c < bc) {
      best = L;
      bc = c;
    }
  }
  return best;
}

// Code forming `name`, the slot of the thread's base index tb in layout L.
void emit_slot_of_tb(Src& o, const char* name, const Layout& L, const uint8_t* rp, int rq) {
  o.line("    uint32_t %s = tb;", name);
  for (int b = 4; b < 12; b++) {
    bool reg = false;
    for (int i = 0; i < rq; i++) reg = reg || rp[i] == b;
    if (!reg && L.col[b - 4]) o.line("    %s ^= (tb & 0x%xu) ? 0x%xu : 0u;", name, 1u << b, L.col[b - 4]);
  }
}

std::string slots_of_bits(const Layout& L, const uint8_t* rp, int rq) {
  std::string ms;
  for (int i = 0; i < rq; i++) ms += (i ? ", " : "") + std::to_string(slot_of(L, 1u << rp[i])) + "u";
  return ms;
}

// The copy of a tile from its stage in shared memory to the state, in 16-byte
// chunks: thread t of the group takes chunks t + 128 k (k < 16), so its local
// bits 1..7 come from t and bits 8..11 from k.  Tile offsets and the swizzle
// are both linear over XOR, so the thread's part is formed once and each
// chunk adds a constant.  L is the layout the tile is in.
void emit_copy_out(Src& o, const ProgramHeader& h, const Layout& L) {
  o.line("  {  // the tile to the state, 16-byte chunks, lanes on consecutive chunks");
  o.line("    uint64_t t0 = 0;");
  for (int b = 0; b < 7; b++) o.line("    t0 |= (uint64_t)((gr.tid >> %d) & 1u) << %d;", b, h.tq[b + 1]);
  o.line("    uint32_t p0 = 0;");
  for (int b = 0; b < 7; b++) o.line("    p0 ^= (gr.tid & 0x%xu) ? 0x%xu : 0u;", 1u << b, slot_of(L, 2u << b));
  for (int k = 0; k < 16; k++) {
    uint64_t go = 0;
    for (int i = 0; i < 4; i++)
      if ((k >> i) & 1) go |= 1ull << h.tq[8 + i];
    const uint32_t pk = slot_of(L, (uint32_t)k << 8);
    o.line("    *reinterpret_cast<uint4*>(state + (base | t0 | 0x%llxull)) = *reinterpret_cast<const uint4*>(s + (p0 ^ %uu));",
           (unsigned long long)go, pk);
  }
  o.line("  }");
}

// The condition of an op on the bits outside the tile and on the thread's
// bits (empty when the op applies everywhere).
std::string op_guard(const DevOp& op, uint32_t code) {
  std::string g;
  char buf[160];
  if (code & (OPF_XCOND << 4)) {
    snprintf(buf, sizeof(buf), "(base & 0x%llxull) == 0x%llxull", (unsigned long long)op.xmask,
             (unsigned long long)op.xval);
    g += buf;
  }
  if (code & (OPF_TCOND << 4)) {
    snprintf(buf, sizeof(buf), "(tb & 0x%xu) == 0x%xu", op.tmask, op.tval);
    if (!g.empty()) g += " && ";
    g += buf;
  }
  return g;
}

// One register op (not a sign flip), as apply_reg of the interpreting kernel
// dispatches it, with every dispatch decision taken here.  Coefficients at an
// offset known here are read from the program in kernel-parameter space
// (`pc`, the constant bank): they are the same for every thread, so they cost
// no shared-memory instruction, and the values are those of the pool copy in
// shared memory (`cf`), which keeps the reads whose offset depends on the
// thread or the tile.
template <typename R>
void emit_reg_op(Src& o, const DevOp& op, int op_index, int rq) {
  const uint32_t code = op.pad;
  const uint32_t kind = code & 15u, fl = (code >> 4) & 7u;
  const uint32_t C = code >> 17, rm = (code >> 7) & 31u, rv = (code >> 12) & 31u;
  const char* Rn = sizeof(R) == 4 ? "float" : "double";
  const std::string g = op_guard(op, code);
  o.line("    %s{  // op %d", g.empty() ? "" : ("if (" + g + ") ").c_str(), op_index);
  switch (kind) {
    case OPK_KRON:
      for (int S = 0; S < rq; S++)
        if (rm & (1u << S)) {
          o.line("      r_u1<%s, %d, %d>(v, pc + %u);", Rn, rq, S, C + 4u * S);
          o.line("      asm volatile(\"\" ::: \"memory\");");
        }
      break;
    case OPK_KROT:
      for (int S = 0; S < rq; S++)
        if (rm & (1u << S)) {
          const bool cot = sizeof(R) == 8 && ((rv >> S) & 1u);
          o.line("      r_rot<%s, %d, %d, %s>(v, pc[%u]);", Rn, rq, S, cot ? "true" : "false", C + S);
          o.line("      asm volatile(\"\" ::: \"memory\");");
        }
      break;
    case OPK_PHASE: {
      std::string var;
      char buf[96];
      for (int i = 0; i < op.k; i++) {
        const uint32_t c = op.gq[i];
        if (c < 64)
          snprintf(buf, sizeof(buf), "(((tb >> %u) & 1u) << %d)", c, i);
        else
          snprintf(buf, sizeof(buf), "((uint32_t)((base >> %u) & 1ull) << %d)", c - 64, i);
        if (!var.empty()) var += " | ";
        var += buf;
      }
      if (var.empty())
        o.line("      r_phase_table<%s, %d>(v, pc + %u);", Rn, rq, C);
      else
        o.line("      r_phase_table<%s, %d>(v, cf + %u + (%s) * %du);", Rn, rq, C, var.c_str(),
               table_stride<R>(rq));
      break;
    }
    case OPK_DENSE:
    case OPK_REAL:
      if (op.k == 1)
        o.line("      r_dense1<%s, %d, %d, %s>(v, pc + %u, 0x%xu, 0x%xu);", Rn, rq, op.rs[0],
               kind == OPK_REAL ? "true" : "false", C, rm, rv);
      else
        o.line("      r_dense2<%s, %d, %d, %d>(v, pc + %u, 0x%xu, 0x%xu);", Rn, rq, op.rs[0], op.rs[1], C, rm, rv);
      break;
    case OPK_ANTIDIAG:
      o.line("      r_anti1<%s, %d, %d, %s>(v, pc + %u, 0x%xu, 0x%xu);", Rn, rq, op.rs[0],
             (fl & OPF_FLIP) ? "true" : "false", C, rm, rv);
      break;
    case OPK_SWAP:
      o.line("      r_swap<%s, %d, %d, %d>(v, 0x%xu, 0x%xu);", Rn, rq, op.rs[0], op.rs[1], rm, rv);
      break;
    case OPK_DIAG:
      o.line("      r_diag<%s, %d>(v, P.ops[%d], cf + %u, tb, base);", Rn, rq, op_index, C);
      break;
    default: break;
  }
  o.line("    }");
}

}  // namespace

// The kernel source of one program (see the top of this file); empty if the
// program is not one the TMA pass runs (complex64, 12-qubit tiles of 128
// threads with five register qubits, at least 2^9 tiles).
template <typename R>
std::string jit_source(const SweepProgram<R>& P) {
  const ProgramHeader& h = P.h;
  const int rq = h.rq;
  if (sizeof(R) != 4 || rq != 5 || (1 << (h.m - rq)) != kJitGroupThreads || h.n - h.m < 9) return std::string();
  const char* Rn = sizeof(R) == 4 ? "float" : "double";
  Src o;
  o.line("// pass program: n %d, m %d, %d phases, %d ops, %d coefficients", h.n, h.m, h.nphases, h.nops, h.ncoef);
  o.line("#include \"sv_tma_pass.cuh\"");
  o.line("namespace sv {");
  o.line("struct alignas(64) JitTensorMap { unsigned long long opaque[16]; };");
  o.line("struct JitRunner {");
  o.line("  const SweepProgram<%s>& P;", Rn);
  o.line("  template <class Release>");
  o.line("  __device__ __forceinline__ void operator()(Cx<%s>* s, const Cx<%s>* cf, uint64_t base, const Grp& gr,", Rn,
         Rn);
  o.line("                                             Cx<%s>* __restrict__ state, const Release& release) const {", Rn);
  o.line("  const Cx<%s>* __restrict__ pc = P.coef;", Rn);
  bool direct_done = false;
  Layout lin = kPhysLayout;  // the layout the next phase finds the tile in
  for (int p = 0; p < h.nphases; p++) {
    const Phase& ph = P.ph[p];
    const bool last = p == h.nphases - 1;
    if (ph.kind == PH_REG) {
      const bool direct = last && direct_store_lines(h, ph, rq) <= kDirectStoreMaxLines;
      const Layout lout = direct                             ? kPhysLayout
                          : last                             ? choose_layout(ph, nullptr, rq)
                          : P.ph[p + 1].kind == PH_REG ? choose_layout(ph, &P.ph[p + 1], rq)
                                                             : kPhysLayout;
      const char* pairs = ph.rp[0] == 0 ? "true" : "false";
      o.line("  {  // phase %d: register slots at local bits %d %d %d %d %d", p, ph.rp[0], ph.rp[1], ph.rp[2],
             ph.rp[3], ph.rp[4]);
      const bool all_active = (1 << ph.ntpos) >= kJitGroupThreads;
      o.line("    uint32_t tb = gr.tid;");
      for (int i = 0; i < rq; i++) o.line("    tb = ins0(tb, %d);", ph.rp[i]);
      std::string ms;
      for (int i = 0; i < rq; i++) ms += (i ? ", " : "") + std::to_string(1u << ph.rp[i]) + "u";
      o.line("    const uint32_t m[%d] = {%s};", rq, ms.c_str());
      o.line("    Cx<%s> v[%d];", Rn, 1 << rq);
      const std::string act = all_active ? "" : "if (gr.tid < " + std::to_string(1u << ph.ntpos) + "u) ";
      emit_slot_of_tb(o, "si", lin, ph.rp, rq);
      o.line("    const uint32_t mi[%d] = {%s};", rq, slots_of_bits(lin, ph.rp, rq).c_str());
      o.line("    %sreg_load_at<%s, %d, %s>(v, s, si, mi);", act.c_str(), Rn, rq, pairs);
      if (direct) {
        o.line("    grp_sync(gr);  // every thread has its registers: the stage is free");
        o.line("    release();");
      }
      o.line("    %s{", act.c_str());
      o.line("    uint32_t neg = 0;");
      for (int i = 0; i < ph.nops; i++) {
        const int oi = ph.first + i;
        const DevOp& op = P.ops[oi];
        const uint32_t code = op.pad;
        if ((code & 15u) == OPK_SIGN) {
          const std::string g = op_guard(op, code);
          if (g.empty())
            o.line("    neg ^= 0x%xu;  // op %d", op.coef, oi);
          else
            o.line("    if (%s) neg ^= 0x%xu;  // op %d", g.c_str(), op.coef, oi);
          continue;
        }
        o.line("    if (neg) { apply_neg<%s, %d>(v, neg); neg = 0; }", Rn, rq);
        emit_reg_op<R>(o, op, oi, rq);
      }
      o.line("    if (neg) apply_neg<%s, %d>(v, neg);", Rn, rq);
      if (direct) {
        std::string gs;
        for (int i = 0; i < rq; i++) gs += (i ? ", " : "") + std::to_string(1ull << h.tq[ph.rp[i]]) + "ull";
        o.line("    const uint64_t gs[%d] = {%s};", rq, gs.c_str());
        // the tile offset of the thread's bits (every local bit outside the
        // register slots): local bit i is global bit tq[i]
        o.line("    uint64_t toff = 0;");
        for (int i = 0; i < h.m; i++) {
          bool reg = false;
          for (int j = 0; j < rq; j++) reg = reg || ph.rp[j] == i;
          if (!reg) o.line("    toff |= (uint64_t)((tb >> %d) & 1u) << %d;", i, h.tq[i]);
        }
        o.line("    reg_store_global<%s, %d>(v, state, base | toff, gs, %s);", Rn, rq, ph.rp[0] == 0 ? "true" : "false");
        direct_done = true;
      } else {
        emit_slot_of_tb(o, "so", lout, ph.rp, rq);
        o.line("    const uint32_t mo[%d] = {%s};", rq, slots_of_bits(lout, ph.rp, rq).c_str());
        o.line("    reg_store_at<%s, %d, %s>(v, s, so, mo);", Rn, rq, pairs);
      }
      o.line("    }");
      o.line("  }");
      if (!direct) o.line("  grp_sync(gr);");
      lin = lout;
    } else {
      const DevOp& op = P.ops[ph.first];
      const uint32_t C = op.coef;
      o.line("  {  // phase %d: op %d in shared memory", p, ph.first);
      char cond[128];
      snprintf(cond, sizeof(cond), "(base & 0x%llxull) == 0x%llxull", (unsigned long long)op.xmask,
               (unsigned long long)op.xval);
      const int tsz = 1 << h.m;
      switch (op.kind) {
        case OPK_DIAG:
        case OPK_SIGN:
          o.line("    if (%s) s_diag<%s>(s, %d, P.ops[%d], cf + %u, base, gr);", cond, Rn, tsz, ph.first, C);
          break;
        case OPK_ANTIDIAG:
        case OPK_SWAP:
          o.line("    if (%s) s_perm<%s>(s, %d, P.ops[%d], cf + %u, gr);", cond, Rn, tsz, ph.first, C);
          break;
        default:
          o.line("    if (%s) s_denseK<%s, %d>(s, %d, P.ops[%d], cf + %u, gr);", cond, Rn, (int)op.k, tsz, ph.first, C);
      }
      o.line("  }");
      o.line("  grp_sync(gr);");
      lin = kPhysLayout;  // the shared-memory ops address the tile through phys()
    }
  }
  if (!direct_done) {
    emit_copy_out(o, h, lin);
    o.line("  grp_sync(gr);");
    o.line("  release();");
  }
  o.line("  }");
  o.line("};");
  o.line("}  // namespace sv");
  const int nc = kJitGroups;
  o.line("extern \"C\" __global__ void __launch_bounds__(%d, 1)", nc * kJitGroupThreads);
  o.line("k_sweep_jit(sv::Cx<%s>* __restrict__ state, const __grid_constant__ sv::JitTensorMap tmap,", Rn);
  o.line("            const __grid_constant__ sv::TmaBoxes bx, const __grid_constant__ sv::SweepProgram<%s> P,", Rn);
  o.line("            int ns, int* status) {");
  o.line("  sv::tma_pass_body<%s, %d, %d>(state, &tmap, bx, P.h, P.coef, ns, status, sv::JitRunner{P});", Rn, nc,
         kJitGroupThreads);
  o.line("}");
  return o.s;
}

template std::string jit_source<float>(const SweepProgram<float>&);
template std::string jit_source<double>(const SweepProgram<double>&);

namespace {

// A BOp as an aggregate initializer, with the fields the tile code reads;
// coef, gen, gidx and table (read once per CTA from the program in parameter
// space) are left zero so that programs differing only there share a kernel.
std::string bop_literal(const BOp& d) {
  char b[512];
  snprintf(b, sizeof(b),
           "{%u, %u, {%u, %u}, {%u, %u}, {%u, %u}, {%u, %u}, 0, %u, %u, %u, %u, %u, 0x%xu, 0x%xu, 0x%xu, 0x%xu, "
           "0x%llxull, 0x%llxull, 0, 0, 0, %u, %u}",
           d.kind, d.k, d.pos[0], d.pos[1], d.spos[0], d.spos[1], d.gq[0], d.gq[1], d.rs[0], d.rs[1], d.dagger, d.grad,
           d.gacc, d.rmask, d.rval, d.lmask, d.lval, d.tmask, d.tval, (unsigned long long)d.xmask,
           (unsigned long long)d.xval, d.flags, d.soff);
  return b;
}

// A register phase as an aggregate initializer (kind, register positions and
// the count of thread positions: what the tile code reads).
std::string phase_literal(const Phase& ph) {
  std::string s = "{" + std::to_string(ph.kind) + ", 0, 0, " + std::to_string(ph.ntpos) + ", " +
                  std::to_string(ph.nrp) + ", {";
  for (int i = 0; i < kMaxRegQ; i++) s += (i ? ", " : "") + std::to_string(ph.rp[i]);
  s += "}, {";
  for (int i = 0; i < kMaxTileQ; i++) s += (i ? ", " : "") + std::to_string(ph.tpos[i]);
  return s + "}}";
}

// The register-op call b_apply (sv_batch_ops.cuh) makes for op d, with its
// dispatch decided here: the function and its template arguments.
std::string batch_reg_call(const BOp& d, bool rev, const char* Rn) {
  const char* RV = rev ? "true" : "false";
  char b[256];
  const bool grad = rev && d.grad;
  const bool plain = d.rmask == 0 && d.rs[0] != 0xFF;
  if (plain && d.k == 1 && (d.kind == OPK_DENSE || d.kind == OPK_REAL)) {
    const bool real = d.flags & OPF_REALM;
    const int gk = !grad ? 0 : (d.flags & OPF_GX) ? 1 : (d.flags & OPF_GY) ? 2 : 3;
    if (gk != 3) {
      const bool r = real && (gk == 2 || gk == 0);
      snprintf(b, sizeof(b), "b_u1<%s, %d, %s, %s, %d>(p, l, op, M, acc);", Rn, d.rs[0] > 3 ? 3 : d.rs[0], RV,
               r ? "true" : "false", gk);
      return b;
    }
  }
  if (plain && d.k == 1 && d.kind == OPK_DIAG) {
    const bool gz = grad && (d.flags & OPF_GZ);
    if (gz || !grad) {
      snprintf(b, sizeof(b), "b_d1<%s, %d, %s, %s>(p, l, op, M, acc);", Rn, d.rs[0] > 3 ? 3 : d.rs[0], RV,
               gz ? "true" : "false");
      return b;
    }
  }
  switch (d.kind) {
    case OPK_DENSE:
    case OPK_REAL:
      if (d.k == 1) {
        snprintf(b, sizeof(b), "b_dense1<%s, %d, %s>(p, l, op, M, G, acc);", Rn, d.rs[0] > 3 ? 3 : d.rs[0], RV);
      } else {
        int A = d.rs[0], B = d.rs[1];
        const int code = A * 4 + B;  // the interpreter's pair switch: unlisted codes take (3, 2)
        if (!(code == 1 || code == 2 || code == 3 || code == 4 || code == 6 || code == 7 || code == 8 || code == 9 ||
              code == 11 || code == 12 || code == 13)) {
          A = 3;
          B = 2;
        }
        snprintf(b, sizeof(b), "b_dense2<%s, %d, %d, %s>(p, l, op, M, G, acc);", Rn, A, B, RV);
      }
      return b;
    case OPK_ANTIDIAG:
      snprintf(b, sizeof(b), "b_anti1<%s, %d, %s, %s>(p, l, op, M);", Rn, d.rs[0] > 3 ? 3 : d.rs[0], RV,
               (d.flags & OPF_FLIP) ? "true" : "false");
      return b;
    case OPK_SWAP: {
      const int a = d.rs[0] < d.rs[1] ? d.rs[0] : d.rs[1], c = d.rs[0] < d.rs[1] ? d.rs[1] : d.rs[0];
      const int code = a * 4 + c;
      const int A = (code == 1 || code == 2 || code == 3) ? 0 : (code == 6 || code == 7) ? 1 : 2;
      const int B = code == 1 ? 1 : (code == 2 || code == 6) ? 2 : 3;
      snprintf(b, sizeof(b), "b_swap<%s, %d, %d, %s>(p, l, op);", Rn, A, B, RV);
      return b;
    }
    case OPK_DIAG:
      snprintf(b, sizeof(b), "b_diag<%s, %s>(p, l, op, M, G, tb, base, acc);", Rn, RV);
      return b;
    default: return "";
  }
}

}  // namespace

// The kernel source of one batched adjoint program: every phase and op as a
// constant, the same tile functions and tile loop as the interpreting kernel.
template <typename R>
std::string jit_batch_source(const BatchProgram<R>& P, bool rev) {
  const BatchHeader& h = P.h;
  const char* Rn = sizeof(R) == 4 ? "float" : "double";
  const char* RV = rev ? "true" : "false";
  Src o;
  o.line("// batched %s program: %d phases, %d ops", rev ? "reverse" : "forward", h.nphases, h.nops);
  o.line("#include \"sv_batch_ops.cuh\"");
  o.line("namespace sv {");
  o.line("struct JitBatchRunner {");
  o.line("  __device__ __forceinline__ void operator()(Cx<%s>* sp, Cx<%s>* sl, int tsz, const Cx<%s>* scoef,", Rn, Rn,
         Rn);
  o.line("                                             uint64_t base, double (*gacc)[8], int warp, int lane) const {");
  for (int p = 0; p < h.nphases; p++) {
    const Phase& ph = P.ph[p];
    if (ph.kind == PH_REG) {
      o.line("  {  // phase %d", p);
      o.line("    const Phase ph = %s;", phase_literal(ph).c_str());
      o.line("    batch_reg_phase<%s, %s>(ph, sp, sl, [&](Cx<%s>(&p)[NR], Cx<%s>(&l)[NR], uint32_t tb, bool active) {",
             Rn, RV, Rn, Rn);
      for (int i = 0; i < ph.nops; i++) {
        // batch_reg_op of the interpreting kernel, its dispatch and
        // conditions decided here
        const BOp& d = P.ops[ph.first + i];
        const int dd = 1 << d.k;
        std::string cond = "active";
        char cb[160];
        if (d.xmask) {
          snprintf(cb, sizeof(cb), " && (base & 0x%llxull) == 0x%llxull", (unsigned long long)d.xmask,
                   (unsigned long long)d.xval);
          cond += cb;
        }
        if (d.tmask) {
          snprintf(cb, sizeof(cb), " && (tb & 0x%xu) == 0x%xu", d.tmask, d.tval);
          cond += cb;
        }
        o.line("      {  // op %d", ph.first + i);
        o.line("        const BOp op = %s;", bop_literal(d).c_str());
        o.line("        %s acc = %s(0);", Rn, Rn);
        o.line("        if (%s) {", cond.c_str());
        o.line("          const Cx<%s>* M = scoef + %u;", Rn, (unsigned)d.soff);
        o.line("          const Cx<%s>* G = M + %d;", Rn, d.kind == OPK_DIAG ? dd : dd * dd);
        o.line("          (void)G;");
        o.line("          %s", batch_reg_call(d, rev, Rn).c_str());
        o.line("        }");
        if (rev && d.grad) o.line("        batch_grad_add<%s>(acc, gacc[%u], warp, lane);", Rn, (unsigned)d.gacc);
        o.line("      }");
      }
      o.line("    });");
      o.line("  }");
    } else {
      o.line("  {  // phase %d, in shared memory", p);
      o.line("    const BOp op = %s;", bop_literal(P.ops[ph.first]).c_str());
      o.line("    batch_smem_op<%s, %s>(op, sp, sl, tsz, scoef, base, gacc, warp, lane);", Rn, RV);
      o.line("  }");
    }
    o.line("  __syncthreads();");
  }
  o.line("  }");
  o.line("};");
  o.line("}  // namespace sv");
  o.line("extern \"C\" __global__ void __launch_bounds__(256, %d)", sizeof(R) == 4 ? 2 : 1);
  o.line("k_batch_sweep_jit(sv::Cx<%s>* __restrict__ psi, sv::Cx<%s>* __restrict__ lam,", Rn, Rn);
  o.line("                  const sv::Cx<%s>* __restrict__ table, double* __restrict__ gscratch,", Rn);
  o.line("                  const __grid_constant__ sv::BatchProgram<%s> P) {", Rn);
  o.line("  sv::batch_sweep_body<%s, %s>(psi, lam, table, gscratch, P, sv::JitBatchRunner{});", Rn, RV);
  o.line("}");
  return o.s;
}

template std::string jit_batch_source<float>(const BatchProgram<float>&, bool);
template std::string jit_batch_source<double>(const BatchProgram<double>&, bool);

namespace {

// ---------------------------------------------------------------- NVRTC

struct Nvrtc {
  bool ok = false;
  std::string why;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
};

const Nvrtc& nvrtc() {
  static Nvrtc n = [] {
    Nvrtc r;
    void* h = nullptr;
    for (const char* name : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"}) {
      h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
      if (h) break;
    }
    if (!h) {
      r.why = "libnvrtc not found";
      return r;
    }
    r.create = (decltype(r.create))dlsym(h, "nvrtcCreateProgram");
    r.compile = (decltype(r.compile))dlsym(h, "nvrtcCompileProgram");
    r.destroy = (decltype(r.destroy))dlsym(h, "nvrtcDestroyProgram");
    r.log_size = (decltype(r.log_size))dlsym(h, "nvrtcGetProgramLogSize");
    r.log = (decltype(r.log))dlsym(h, "nvrtcGetProgramLog");
    r.cubin_size = (decltype(r.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
    r.cubin = (decltype(r.cubin))dlsym(h, "nvrtcGetCUBIN");
    r.ok = r.create && r.compile && r.destroy && r.log_size && r.log && r.cubin_size && r.cubin;
    if (!r.ok) r.why = "libnvrtc lacks an entry point";
    return r;
  }();
  return n;
}

// Compiles one kernel source to a cubin for sm_<arch>; false with the
// compiler's log in *log on failure.
bool compile_cubin(const std::string& src, int arch, std::vector<char>& out, std::string* log) {
  const Nvrtc& nv = nvrtc();
  if (!nv.ok) {
    if (log) *log = nv.why;
    return false;
  }
  constexpr int NH = sizeof(kJitHeaderNames) / sizeof(kJitHeaderNames[0]);
  nvrtcProgram prog = nullptr;
  if (nv.create(&prog, src.c_str(), "sv_pass.cu", NH, kJitHeaderTexts, kJitHeaderNames) != NVRTC_SUCCESS) {
    if (log) *log = "nvrtcCreateProgram failed";
    return false;
  }
  const std::string archopt = "--gpu-architecture=sm_" + std::to_string(arch) + "a";
  // -default-device: the program-layout header's constexpr helpers are
  // plain functions (host and device in the library's own build)
  const char* opts[] = {archopt.c_str(), "-std=c++17", "-default-device"};
  const nvrtcResult r = nv.compile(prog, 3, opts);
  bool ok = r == NVRTC_SUCCESS;
  if (!ok && log) {
    size_t n = 0;
    nv.log_size(prog, &n);
    std::string l(n, '\0');
    if (n) nv.log(prog, &l[0]);
    *log = l;
  }
  if (ok) {
    size_t n = 0;
    ok = nv.cubin_size(prog, &n) == NVRTC_SUCCESS && n > 0;
    if (ok) {
      out.resize(n);
      ok = nv.cubin(prog, out.data()) == NVRTC_SUCCESS;
    }
  }
  nv.destroy(&prog);
  return ok;
}

// ---------------------------------------------------------------- driver

using ModuleLoadDataFn = CUresult (*)(CUmodule*, const void*);
using ModuleGetFunctionFn = CUresult (*)(CUfunction*, CUmodule, const char*);
using FuncSetAttributeFn = CUresult (*)(CUfunction, CUfunction_attribute, int);
using FuncGetAttributeFn = CUresult (*)(int*, CUfunction_attribute, CUfunction);
using LaunchKernelFn = CUresult (*)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                                    CUstream, void**, void**);

struct Driver {
  bool ok = false;
  ModuleLoadDataFn load = nullptr;
  ModuleGetFunctionFn get = nullptr;
  FuncSetAttributeFn attr = nullptr;
  FuncGetAttributeFn getattr = nullptr;
  LaunchKernelFn launch = nullptr;
};

template <typename F>
F entry(const char* name) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (F)p;
}

const Driver& driver() {
  static Driver d = [] {
    Driver r;
    r.load = entry<ModuleLoadDataFn>("cuModuleLoadData");
    r.get = entry<ModuleGetFunctionFn>("cuModuleGetFunction");
    r.attr = entry<FuncSetAttributeFn>("cuFuncSetAttribute");
    r.getattr = entry<FuncGetAttributeFn>("cuFuncGetAttribute");
    r.launch = entry<LaunchKernelFn>("cuLaunchKernel");
    r.ok = r.load && r.get && r.attr && r.getattr && r.launch;
    return r;
  }();
  return d;
}

// ---------------------------------------------------------------- cache and policy

std::mutex g_jit_mu;
std::map<std::pair<int, std::string>, std::unique_ptr<JitKernel>> g_jit_kernels;  // (device, source) -> kernel
std::atomic<int> g_jit_mode{-1};
std::atomic<long long> g_jit_compiled{0}, g_jit_failed{0}, g_jit_launches{0};
std::atomic<long long> g_jit_compile_us{0};
std::string g_jit_last_error;

int device_arch(int dev) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major * 10 + minor;
}

// Compiles in flight across the process: callers on several threads (the
// workers of a serving loop) share one budget of host cores.
std::mutex g_slots_mu;
std::condition_variable g_slots_cv;
int g_slots_used = 0;

int compile_slots() {
  static const int n = [] {
    const unsigned hw = std::thread::hardware_concurrency();
    return (int)(hw ? std::min(hw, 16u) : 4u);
  }();
  return n;
}

// Compiles the given sources in parallel (host threads; NVRTC needs no
// device), each to a cubin, at most compile_slots() at a time in the process.
void compile_all(const std::vector<const std::string*>& srcs, int arch, std::vector<std::vector<char>>& bins,
                 std::vector<std::string>& logs, std::vector<char>& ok) {
  const size_t n = srcs.size();
  bins.assign(n, {});
  logs.assign(n, {});
  ok.assign(n, 0);
  std::atomic<size_t> next{0};
  auto work = [&] {
    for (size_t i; (i = next.fetch_add(1)) < n;) {
      {
        std::unique_lock<std::mutex> lk(g_slots_mu);
        g_slots_cv.wait(lk, [] { return g_slots_used < compile_slots(); });
        g_slots_used++;
      }
      ok[i] = compile_cubin(*srcs[i], arch, bins[i], &logs[i]) ? 1 : 0;
      {
        std::lock_guard<std::mutex> lk(g_slots_mu);
        g_slots_used--;
      }
      g_slots_cv.notify_one();
    }
  };
  const size_t nt = std::min<size_t>(n, (size_t)compile_slots());
  std::vector<std::thread> th;
  for (size_t t = 1; t < nt; t++) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
}

}  // namespace

int jit_mode() {
  int m = g_jit_mode.load();
  if (m < 0) {
    const char* e = std::getenv("SV_JIT");
    m = 1;
    if (e && e[0] == '0') m = 0;
    if (e && (e[0] == '2' || std::strcmp(e, "eager") == 0)) m = 2;
    g_jit_mode.store(m);
  }
  return m;
}

void jit_set_mode(int mode) { g_jit_mode.store(mode < 0 ? -1 : mode); }

namespace {

// Kernels for the given sources (empty: none) on the current device, named
// `name` in their modules: compiles, in parallel, the distinct sources the
// cache lacks, then loads them.  NULL where a source is empty or failed.
std::vector<const JitKernel*> kernels_for(const std::vector<std::string>& src, const char* name) {
  std::vector<const JitKernel*> out(src.size(), nullptr);
  if (!driver().ok || !nvrtc().ok) return out;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return out;
  }
  const int arch = device_arch(dev);
  std::vector<const std::string*> todo;
  {
    std::lock_guard<std::mutex> lk(g_jit_mu);
    std::map<std::string, size_t> seen;
    for (size_t i = 0; i < src.size(); i++) {
      if (src[i].empty()) continue;
      auto it = g_jit_kernels.find({dev, src[i]});
      if (it != g_jit_kernels.end()) {
        out[i] = it->second.get();
        continue;
      }
      if (seen.emplace(src[i], i).second) todo.push_back(&src[i]);
    }
  }
  if (todo.empty()) return out;
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<std::vector<char>> bins;
  std::vector<std::string> logs;
  std::vector<char> ok;
  compile_all(todo, arch, bins, logs, ok);
  g_jit_compile_us +=
      (long long)std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
  // a module load waits for every resident kernel of the device, so the
  // device's serving sessions are paused around the loads
  struct Pause {
    std::vector<sv_small_session*> held;
    explicit Pause(int d) { sessions_quiesce(d, held); }
    ~Pause() { sessions_release(held); }
  };
  {
    Pause pause(dev);
    std::lock_guard<std::mutex> lk(g_jit_mu);
    for (size_t t = 0; t < todo.size(); t++) {
      if (!ok[t]) {
        g_jit_failed++;
        g_jit_last_error = logs[t].substr(0, 4000);
        continue;
      }
      // another thread may have compiled and loaded the same source meanwhile:
      // its kernel stays (callers may hold it), this one is not loaded
      if (g_jit_kernels.count({dev, *todo[t]})) continue;
      CUmodule mod = nullptr;
      auto k = std::make_unique<JitKernel>();
      if (driver().load(&mod, bins[t].data()) != CUDA_SUCCESS || driver().get(&k->fn, mod, name) != CUDA_SUCCESS) {
        g_jit_failed++;
        g_jit_last_error = "module load failed";
        continue;
      }
      // the dynamic shared memory a launch may ask for, set here while the
      // sessions are paused: the block's opt-in limit less the kernel's own
      // static shared memory (a launch asking for more sets it again)
      int stat = 0, optin = 0;
      if (driver().getattr(&stat, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, k->fn) == CUDA_SUCCESS &&
          cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
          optin > stat &&
          driver().attr(k->fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, optin - stat) == CUDA_SUCCESS)
        k->smem_configured.store((size_t)(optin - stat));
      cudaGetLastError();
      k->device = dev;
      g_jit_compiled++;
      g_jit_kernels.emplace(std::make_pair(dev, *todo[t]), std::move(k));
    }
  }
  std::lock_guard<std::mutex> lk(g_jit_mu);
  for (size_t i = 0; i < src.size(); i++) {
    if (out[i] || src[i].empty()) continue;
    auto it = g_jit_kernels.find({dev, src[i]});
    if (it != g_jit_kernels.end()) out[i] = it->second.get();
  }
  return out;
}

// Batched programs: (device, direction, precision, the op and phase bytes) ->
// kernel, so that a launch finds its kernel without writing the source.
std::unordered_map<std::string, const JitKernel*> g_batch_kernels;

template <typename R>
std::string batch_key(const BatchProgram<R>& P, bool rev, int dev) {
  std::string k;
  const int32_t hdr[4] = {dev, rev ? 1 : 0, (int32_t)sizeof(R), P.h.nphases};
  k.append((const char*)hdr, sizeof(hdr));
  k.append((const char*)P.ops, sizeof(BOp) * (size_t)P.h.nops);
  k.append((const char*)P.ph, sizeof(Phase) * (size_t)P.h.nphases);
  return k;
}

}  // namespace

template <typename R>
std::vector<const JitKernel*> jit_compile_programs(const std::vector<SweepProgram<R>>& progs) {
  std::vector<std::string> src(progs.size());
  if (sizeof(R) == 4)
    for (size_t i = 0; i < progs.size(); i++) src[i] = jit_source<R>(progs[i]);
  return kernels_for(src, "k_sweep_jit");
}

// ---- pass programs keyed by structure
//
// A program's key is everything its kernel source is written from -- the
// header (sizes, tile qubits, pool size), its ops and its phases -- and none
// of its coefficient values, so every circuit of the same structure (the same
// gates at other angles: a variational template, the requests of a serving
// family) shares the kernel.  Uses are counted per key (by a 64-bit hash, in a
// table cleared when it grows past a million keys); a key reaching the
// threshold is compiled in the calling thread, together with the call's other
// keys that reached it.

namespace {

std::unordered_map<std::string, const JitKernel*> g_key_kernels;  // device + key -> kernel
std::unordered_map<uint64_t, int> g_key_uses;                     // hash(device + key) -> uses

uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : s) h = (h ^ c) * 1099511628211ull;
  return h;
}

}  // namespace

std::string jit_program_key(const SweepProgram<float>& P) {
  const ProgramHeader& h = P.h;
  if (h.rq != 5 || (1 << (h.m - h.rq)) != kJitGroupThreads || h.n - h.m < 9) return std::string();
  std::string k;
  const int32_t hdr[7] = {h.n, h.m, h.L, h.nops, h.ncoef, h.nphases, h.rq};
  k.append((const char*)hdr, sizeof(hdr));
  k.append((const char*)h.tq, sizeof(h.tq));
  k.append((const char*)P.ops, sizeof(DevOp) * (size_t)h.nops);
  k.append((const char*)P.ph, sizeof(Phase) * (size_t)h.nphases);
  return k;
}

std::vector<const JitKernel*> jit_program_kernels(const std::vector<SweepProgram<float>>& progs,
                                                  const std::vector<std::string>& keys, int threshold) {
  std::vector<const JitKernel*> out(progs.size(), nullptr);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return out;
  }
  const std::string tag((const char*)&dev, sizeof(dev));
  std::vector<size_t> want;
  {
    std::lock_guard<std::mutex> lk(g_jit_mu);
    if (g_key_uses.size() > (1u << 20)) g_key_uses.clear();
    for (size_t i = 0; i < progs.size() && i < keys.size(); i++) {
      if (keys[i].empty()) continue;
      const std::string full = tag + keys[i];
      auto it = g_key_kernels.find(full);
      if (it != g_key_kernels.end()) {
        out[i] = it->second;
        continue;
      }
      if (++g_key_uses[fnv1a(full)] >= threshold) want.push_back(i);
    }
  }
  if (want.empty() || !driver().ok || !nvrtc().ok) return out;
  std::vector<std::string> src(want.size());
  for (size_t j = 0; j < want.size(); j++) src[j] = jit_source<float>(progs[want[j]]);
  const std::vector<const JitKernel*> k = kernels_for(src, "k_sweep_jit");
  std::lock_guard<std::mutex> lk(g_jit_mu);
  for (size_t j = 0; j < want.size(); j++) {
    if (!k[j]) continue;
    g_key_kernels[tag + keys[want[j]]] = k[j];
    out[want[j]] = k[j];
  }
  return out;
}

template <typename R>
void jit_batch_prepare(const std::vector<const BatchProgram<R>*>& progs, const std::vector<char>& rev) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  std::vector<std::string> src(progs.size()), keys(progs.size());
  {
    std::lock_guard<std::mutex> lk(g_jit_mu);
    for (size_t i = 0; i < progs.size(); i++) {
      keys[i] = batch_key<R>(*progs[i], rev[i] != 0, dev);
      if (!g_batch_kernels.count(keys[i])) src[i] = jit_batch_source<R>(*progs[i], rev[i] != 0);
    }
  }
  std::vector<const JitKernel*> k = kernels_for(src, "k_batch_sweep_jit");
  std::lock_guard<std::mutex> lk(g_jit_mu);
  for (size_t i = 0; i < progs.size(); i++)
    if (k[i]) g_batch_kernels[keys[i]] = k[i];
}

template <typename R>
const JitKernel* jit_batch_lookup(const BatchProgram<R>& P, bool rev) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const std::string key = batch_key<R>(P, rev, dev);
  std::lock_guard<std::mutex> lk(g_jit_mu);
  auto it = g_batch_kernels.find(key);
  return it == g_batch_kernels.end() ? nullptr : it->second;
}

template void jit_batch_prepare<float>(const std::vector<const BatchProgram<float>*>&, const std::vector<char>&);
template void jit_batch_prepare<double>(const std::vector<const BatchProgram<double>*>&, const std::vector<char>&);
template const JitKernel* jit_batch_lookup<float>(const BatchProgram<float>&, bool);
template const JitKernel* jit_batch_lookup<double>(const BatchProgram<double>&, bool);

namespace {

// Raises a kernel's dynamic shared-memory allowance to `smem` if it is below
// (normally set at load to the block's limit, so this is rare); raises are
// serialized so that concurrent launches never lower it.
std::mutex g_smem_mu;
bool allow_smem(JitKernel* k, size_t smem) {
  if (smem <= k->smem_configured.load(std::memory_order_acquire)) return true;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  if (smem <= k->smem_configured.load(std::memory_order_acquire)) return true;
  if (smem > 48 * 1024 &&
      driver().attr(k->fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)smem) != CUDA_SUCCESS)
    return false;
  k->smem_configured.store(smem, std::memory_order_release);
  return true;
}

}  // namespace

cudaError_t jit_batch_launch(const JitKernel* k, void* psi, void* lam, const void* table, double* gscratch,
                             const void* prog, unsigned grid_x, unsigned batch, unsigned threads, size_t smem,
                             cudaStream_t stream) {
  const Driver& d = driver();
  int dev = 0;
  cudaGetDevice(&dev);
  if (!k || !k->fn || k->device != dev) return cudaErrorInvalidDeviceFunction;
  if (!allow_smem(const_cast<JitKernel*>(k), smem)) return cudaErrorInvalidConfiguration;
  JitKernel* kk = const_cast<JitKernel*>(k);
  void* a0 = psi;
  void* a1 = lam;
  const void* a2 = table;
  double* a3 = gscratch;
  void* args[] = {&a0, &a1, &a2, &a3, const_cast<void*>(prog)};
  const CUresult r = d.launch(kk->fn, grid_x, batch, 1, threads, 1, 1, (unsigned)smem, (CUstream)stream, args, nullptr);
  if (r != CUDA_SUCCESS) return cudaErrorLaunchFailure;
  g_jit_launches++;
  return cudaSuccess;
}

// Writes (and with compile, compiles) the kernels of the given batched
// programs without a device.
template <typename R>
void jit_check_batch(const std::vector<const BatchProgram<R>*>& progs, const std::vector<char>& rev, bool compile,
                     int arch, int* n_sources, int* n_compiled, std::string* first_error, std::string* sources) {
  std::vector<std::string> src;
  std::map<std::string, int> seen;
  for (size_t i = 0; i < progs.size(); i++) {
    std::string s = jit_batch_source<R>(*progs[i], rev[i] != 0);
    if (seen.emplace(s, 1).second) src.push_back(std::move(s));
  }
  *n_sources = (int)src.size();
  *n_compiled = 0;
  if (sources)
    for (const std::string& s : src) *sources += s + "// ----\n";
  if (!compile || src.empty()) return;
  std::vector<const std::string*> ptrs;
  for (auto& s : src) ptrs.push_back(&s);
  std::vector<std::vector<char>> bins;
  std::vector<std::string> logs;
  std::vector<char> ok;
  compile_all(ptrs, arch, bins, logs, ok);
  for (size_t i = 0; i < src.size(); i++) {
    if (ok[i])
      (*n_compiled)++;
    else if (first_error && first_error->empty())
      *first_error = logs[i].empty() ? std::string("compile failed") : logs[i];
  }
}

template void jit_check_batch<float>(const std::vector<const BatchProgram<float>*>&, const std::vector<char>&, bool,
                                     int, int*, int*, std::string*, std::string*);
template void jit_check_batch<double>(const std::vector<const BatchProgram<double>*>&, const std::vector<char>&,
                                      bool, int, int*, int*, std::string*, std::string*);

template std::vector<const JitKernel*> jit_compile_programs<float>(const std::vector<SweepProgram<float>>&);
template std::vector<const JitKernel*> jit_compile_programs<double>(const std::vector<SweepProgram<double>>&);

cudaError_t jit_launch(const JitKernel* k, void* state, const void* map, const void* bx, const void* prog, int ns,
                       int* status, unsigned grid, unsigned block, size_t smem, cudaStream_t stream) {
  const Driver& d = driver();
  int dev = 0;
  cudaGetDevice(&dev);
  if (!k || !k->fn || k->device != dev) return cudaErrorInvalidDeviceFunction;
  if (!allow_smem(const_cast<JitKernel*>(k), smem)) return cudaErrorInvalidConfiguration;
  JitKernel* kk = const_cast<JitKernel*>(k);
  void* state_arg = state;
  void* args[] = {&state_arg, const_cast<void*>(map), const_cast<void*>(bx), const_cast<void*>(prog), &ns, &status};
  const CUresult r = d.launch(kk->fn, grid, 1, 1, block, 1, 1, (unsigned)smem, (CUstream)stream, args, nullptr);
  if (r != CUDA_SUCCESS) return cudaErrorLaunchFailure;
  g_jit_launches++;
  return cudaSuccess;
}

// Generates (and with compile set, compiles for sm_<arch>) the kernel of every
// program of a plan without a device (*sources: every source, each followed by
// a "// ----" line): the generator and the run-time
// compiler can be checked on a machine without a GPU.
template <typename R>
void jit_check_programs(const std::vector<SweepProgram<R>>& progs, bool compile, int arch, int* n_sources,
                        int* n_compiled, std::string* first_error, std::string* sources) {
  std::vector<std::string> src;
  for (const auto& P : progs) {
    std::string s = jit_source<R>(P);
    if (!s.empty()) src.push_back(std::move(s));
  }
  *n_sources = (int)src.size();
  *n_compiled = 0;
  if (sources)
    for (const std::string& s : src) *sources += s + "// ----\n";
  if (!compile || src.empty()) return;
  std::vector<const std::string*> ptrs;
  for (auto& s : src) ptrs.push_back(&s);
  std::vector<std::vector<char>> bins;
  std::vector<std::string> logs;
  std::vector<char> ok;
  compile_all(ptrs, arch, bins, logs, ok);
  for (size_t i = 0; i < src.size(); i++) {
    if (ok[i])
      (*n_compiled)++;
    else if (first_error && first_error->empty())
      *first_error = logs[i].empty() ? std::string("compile failed") : logs[i];
  }
}

template void jit_check_programs<float>(const std::vector<SweepProgram<float>>&, bool, int, int*, int*,
                                        std::string*, std::string*);
template void jit_check_programs<double>(const std::vector<SweepProgram<double>>&, bool, int, int*, int*,
                                         std::string*, std::string*);

void jit_stats(long long* compiled, long long* failed, long long* launches, double* compile_seconds,
               std::string* last_error) {
  if (compiled) *compiled = g_jit_compiled.load();
  if (failed) *failed = g_jit_failed.load();
  if (launches) *launches = g_jit_launches.load();
  if (compile_seconds) *compile_seconds = 1e-6 * (double)g_jit_compile_us.load();
  if (last_error) {
    std::lock_guard<std::mutex> lk(g_jit_mu);
    *last_error = g_jit_last_error;
  }
}

bool jit_available(std::string* why) {
  if (!nvrtc().ok) {
    if (why) *why = nvrtc().why;
    return false;
  }
  return true;
}

}  // namespace sv
