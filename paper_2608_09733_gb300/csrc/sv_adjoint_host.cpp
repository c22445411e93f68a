// sv_adjoint_host.cpp -- sv_adjoint_grad: batched adjoint gradients with
// state checkpoints.
//
// For each of B parameter vectors of one circuit template (Sec. 4.2: the
// structure stays fixed while the parameter values change):
//   1. forward pass psi = U_N .. U_1 |0>, storing psi after every
//      `checkpoint_every` gates;
//   2. lambda = H psi with H = sum_j c_j P_j applied matrix-free (Sec. 4.4);
//      f = Re <psi|lambda>;
//   3. reverse pass over the gates: each rotation adds Im <lambda|G|psi> to its
//      slot's gradient, then psi and lambda are un-applied; at a checkpoint
//      boundary psi is replaced by the stored forward state, so complex64
//      uncompute drift never accumulates over more than `checkpoint_every`
//      gates.  (The paper's own checkpointing discards and recomputes states,
//      Sec. 7.3; here stored states re-anchor the uncompute.)
// Per-state gate matrices are built on the host in double precision and
// narrowed once (Sec. 3.3, Sec. 5.2).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <memory>

#include "sv_adjoint.h"

namespace sv {
namespace {

bool is_rotation(int t) {
  return t == SV_GATE_RX || t == SV_GATE_RY || t == SV_GATE_RZ || t == SV_GATE_P || t == SV_GATE_RXX ||
         t == SV_GATE_RYY || t == SV_GATE_RZZ || t == SV_GATE_EXC1 || t == SV_GATE_EXC2;
}
bool rotation_is_diagonal(int t) { return t == SV_GATE_RZ || t == SV_GATE_P || t == SV_GATE_RZZ; }

// Generator G of U = exp(-i theta G / 2) on the targets: dense d x d, or the
// d diagonal entries for the diagonal families.
std::vector<cplx> generator_of(int t) {
  const cplx j(0.0, 1.0);
  switch (t) {
    case SV_GATE_RX: return {0.0, 1.0, 1.0, 0.0};
    case SV_GATE_RY: return {0.0, -j, j, 0.0};
    case SV_GATE_RZ: return {1.0, -1.0};
    case SV_GATE_P: return {0.0, -2.0};  // diag(1, e^{i t}) = exp(-i t (Z - I) / 2)
    case SV_GATE_RZZ: return {1.0, -1.0, -1.0, 1.0};
    case SV_GATE_RXX: {
      std::vector<cplx> m(16, 0.0);
      m[0 * 4 + 3] = m[1 * 4 + 2] = m[2 * 4 + 1] = m[3 * 4 + 0] = 1.0;
      return m;
    }
    case SV_GATE_RYY: {
      std::vector<cplx> m(16, 0.0);
      m[0 * 4 + 3] = m[3 * 4 + 0] = -1.0;
      m[1 * 4 + 2] = m[2 * 4 + 1] = 1.0;
      return m;
    }
    case SV_GATE_EXC1: {  // Y on the pair (|10>, |01>) = indices (1, 2)
      std::vector<cplx> m(16, 0.0);
      m[1 * 4 + 2] = -j;
      m[2 * 4 + 1] = j;
      return m;
    }
    default: return {};
  }
}

struct AGate {
  LOp op;               // kind / qubits / controls; m = U for constant gates
  bool param = false;
  int slot = -1;
  int pidx = -1;        // index among the parameterised gates
  std::vector<cplx> gen;
  sv_gate rec;          // the record its matrix is built from
};

// The adjoint takes gates of at most two targets.  A double excitation
// EXC2(theta) on (t0, t1, t2, t3) rotates the pair of basis states t0 t1 set /
// t2 t3 set (matrix indices 3 and 12) and leaves the rest alone.  The
// permutation C = X(t0) CNOT(t0 -> t2) CNOT(t2 -> t3) CNOT(t0 -> t1) (the
// rightmost first) sends that pair to the two states with t1 = 0, t2 = 1,
// t3 = 0 that differ in t0 (index 3 to t0 = 0, index 12 to t0 = 1) and no
// other state there, so
//   EXC2(theta) = C^dag RY(theta)[t0 | t1 = 0, t2 = 1, t3 = 0] C,
// a controlled one-qubit rotation with generator Y whose gradient term the
// adjoint already takes (the EXC2's own controls join the rotation's).
// Appends the lowering of g to `out`; false when the rotation would need more
// than SV_MAX_CONTROLS controls.
bool expand_gate(const sv_gate& g, std::vector<sv_gate>& out) {
  if (g.type != SV_GATE_EXC2) {
    out.push_back(g);
    return true;
  }
  if (g.n_controls + 3 > SV_MAX_CONTROLS) return false;
  const int t0 = g.targets[0], t1 = g.targets[1], t2 = g.targets[2], t3 = g.targets[3];
  auto fixed = [](int type, int target, int control) {
    sv_gate f;
    std::memset(&f, 0, sizeof(f));
    f.type = type;
    f.n_targets = 1;
    f.targets[0] = target;
    if (control >= 0) {
      f.n_controls = 1;
      f.controls[0] = control;
    }
    f.param_slot[0] = f.param_slot[1] = f.param_slot[2] = -1;
    return f;
  };
  const sv_gate perm[4] = {fixed(SV_GATE_X, t1, t0), fixed(SV_GATE_X, t3, t2), fixed(SV_GATE_X, t2, t0),
                           fixed(SV_GATE_X, t0, -1)};
  for (int k = 0; k < 4; k++) out.push_back(perm[k]);
  sv_gate ry = g;
  ry.type = SV_GATE_RY;
  ry.n_targets = 1;
  ry.targets[0] = t0;
  ry.n_controls = 3 + g.n_controls;
  ry.controls[0] = t1;
  ry.controls[1] = t2;
  ry.controls[2] = t3;
  for (int c = 0; c < g.n_controls; c++) ry.controls[3 + c] = g.controls[c];
  ry.control_zero_mask = 1u | 4u | (g.control_zero_mask << 3);  // t1 = 0, t2 = 1, t3 = 0
  out.push_back(ry);
  for (int k = 3; k >= 0; k--) out.push_back(perm[k]);
  return true;
}

// A circuit template lowered for the adjoint: gate i becomes ag[start[i]] ..
// ag[start[i+1]-1] (one gate, or the nine of a double excitation); npg
// parameterised gates.  Segments and checkpoints count the caller's gates.
struct AdjTemplate {
  std::vector<size_t> start;
  std::vector<AGate> ag;
  int npg = 0;
};

AdjTemplate lower_template(const sv_gate* gates, size_t ng) {
  AdjTemplate T;
  // ---- lower the template: gate i becomes ag[start[i]] .. ag[start[i+1]-1]
  // (one gate, or the nine of a double excitation); segments and checkpoints
  // count the caller's gates
  std::vector<sv_gate> eg;
  std::vector<size_t>& start = T.start;
  start.assign(ng + 1, 0);
  eg.reserve(ng);
  for (size_t i = 0; i < ng; i++) {
    start[i] = eg.size();
    if (!expand_gate(gates[i], eg))
      fail(SV_ERR_UNSUPPORTED, "gate " + std::to_string(i) + ": a double excitation in the adjoint takes at most " +
                                   std::to_string(SV_MAX_CONTROLS - 3) + " controls");
  }
  start[ng] = eg.size();
  std::vector<AGate>& ag = T.ag;
  ag.resize(eg.size());
  int& npg = T.npg;
  npg = 0;
  for (size_t i = 0; i < eg.size(); i++) {
    const sv_gate& g = eg[i];
    ag[i].rec = g;
    bool any_slot = false;
    const int nang = g.type == SV_GATE_U3 ? 3 : g.type == SV_GATE_U2 ? 2 : is_rotation(g.type) ? 1 : 0;
    for (int a = 0; a < nang; a++)
      if (g.param_slot[a] >= 0) any_slot = true;
    const size_t src = (size_t)(std::upper_bound(start.begin(), start.end(), i) - start.begin()) - 1;
    if (g.n_targets > 2)
      fail(SV_ERR_UNSUPPORTED, "gate " + std::to_string(src) + ": the adjoint path takes gates of <= 2 targets "
                                                               "(double excitations aside)");
    AGate& a = ag[i];
    if (any_slot) {
      if (!is_rotation(g.type) || g.param_slot[0] < 0)
        fail(SV_ERR_UNSUPPORTED, "gate " + std::to_string(src) +
                                     ": a parameterised gate needs a generator, exp(-i theta G / 2) "
                                     "(RX, RY, RZ, P, RXX, RYY, RZZ, EXC1, EXC2)");
      a.param = true;
      a.slot = g.param_slot[0];
      a.pidx = npg++;
      a.gen = generator_of(g.type);
      LOp& op = a.op;
      op.k = g.n_targets;
      for (int t = 0; t < op.k; t++) op.q[t] = g.targets[t];
      op.nc = g.n_controls;
      for (int c = 0; c < op.nc; c++) {
        op.c[c] = g.controls[c];
        op.cs[c] = ((g.control_zero_mask >> c) & 1u) ? 0 : 1;
      }
      op.kind = rotation_is_diagonal(g.type) ? OPK_DIAG : OPK_DENSE;
      op.touch = 0;
      uint64_t tm = 0;
      for (int t = 0; t < op.k; t++) tm |= 1ull << op.q[t];
      for (int c = 0; c < op.nc; c++) op.touch |= 1ull << op.c[c];
      op.touch |= tm;
      op.need = op.kind == OPK_DIAG ? 0 : tm;
      op.m.assign(op.kind == OPK_DIAG ? (1 << op.k) : (1 << (2 * op.k)), 0.0);  // sizes the pool use
    } else {
      a.op = lower_gate(g, nullptr, (int)src);
      if (a.op.kind == OPK_REAL) a.op.kind = OPK_DENSE;
    }
    a.op.first_gate = (int)src;
  }

  return T;
}

template <typename R>
void fill_program(const std::vector<AGate>& ag, const std::vector<int>& order, const Sweep& sw, int n, int batch,
                  int npg, bool reverse, BatchProgram<R>& P) {
  std::memset(&P.h, 0, sizeof(P.h));
  P.h.n = n;
  P.h.m = sw.m;
  P.h.L = sw.L;
  P.h.batch = batch;
  P.h.ngrad_total = npg;
  int loc[64];
  for (int q = 0; q < 64; q++) loc[q] = -1;
  for (int i = 0; i < sw.m; i++) {
    P.h.tq[i] = (int8_t)sw.tq[i];
    loc[sw.tq[i]] = i;
  }
  int pool = 0, nacc = 0;
  auto put = [&](const std::vector<cplx>& v) {
    int at = pool;
    for (const cplx& c : v) {
      if (pool >= BatchProgram<R>::kPool) fail(SV_ERR_INVALID, "internal: batch program pool overflow");
      P.pool[pool].re = (R)c.real();
      P.pool[pool].im = (R)c.imag();
      pool++;
    }
    return at;
  };
  if ((int)sw.ops.size() > kBatchOps) fail(SV_ERR_INVALID, "internal: too many ops in a batch program");
  std::vector<uint32_t> need(sw.ops.size(), 0);
  for (size_t oi = 0; oi < sw.ops.size(); oi++) {
    const AGate& g = ag[order[sw.ops[oi]]];
    const LOp& op = g.op;
    BOp d;
    std::memset(&d, 0, sizeof(d));
    d.kind = op.kind;
    d.k = (uint8_t)op.k;
    d.rs[0] = d.rs[1] = 0xFF;
    int sp[2], ns = 0;
    for (int i = 0; i < op.k; i++) {
      int l = loc[op.q[i]];
      d.gq[i] = (uint8_t)op.q[i];
      if (op.kind == OPK_DIAG) {
        d.pos[i] = l < 0 ? 0xFF : (uint8_t)l;
      } else {
        if (l < 0) fail(SV_ERR_INVALID, "internal: target outside the tile");
        d.pos[i] = (uint8_t)l;
        sp[ns++] = l;
        need[oi] |= 1u << l;
      }
    }
    if (ns == 2 && sp[0] > sp[1]) std::swap(sp[0], sp[1]);
    for (int i = 0; i < ns; i++) d.spos[i] = (uint8_t)sp[i];
    for (int i = 0; i < op.nc; i++) {
      int l = loc[op.c[i]];
      if (l >= 0) {
        d.lmask |= 1u << l;
        if (op.cs[i]) d.lval |= 1u << l;
      } else {
        d.xmask |= 1ull << op.c[i];
        if (op.cs[i]) d.xval |= 1ull << op.c[i];
      }
    }
    d.dagger = reverse ? 1 : 0;
    if (op.kind == OPK_ANTIDIAG && op.m.size() == 2 && op.m[0] == cplx(1.0) && op.m[1] == cplx(1.0))
      d.flags |= OPF_FLIP;
    if (g.param) {
      // RY has real matrices; RX, RY, RZ have Pauli generators
      const std::vector<cplx>& G = g.gen;
      const cplx j(0.0, 1.0);
      if (op.k == 1 && op.kind == OPK_DENSE && G == std::vector<cplx>{0.0, -j, j, 0.0}) d.flags |= OPF_REALM | OPF_GY;
      if (op.k == 1 && op.kind == OPK_DENSE && G == std::vector<cplx>{0.0, 1.0, 1.0, 0.0}) d.flags |= OPF_GX;
      if (op.k == 1 && op.kind == OPK_DIAG && G == std::vector<cplx>{1.0, -1.0}) d.flags |= OPF_GZ;
      d.table = 1;
      d.coef = (uint32_t)g.pidx;
      if (reverse) {
        if (nacc >= kBatchGacc) fail(SV_ERR_INVALID, "internal: too many gradient ops in a program");
        d.grad = 1;
        d.gacc = (uint8_t)nacc++;
        d.gidx = (uint32_t)g.pidx;
        d.gen = (uint32_t)put(g.gen);
      }
    } else {
      bool real = op.kind == OPK_DENSE;
      for (const cplx& v : op.m) real = real && v.imag() == 0.0;
      if (real) d.flags |= OPF_REALM;
      d.coef = (uint32_t)put(op.m);
    }
    P.ops[oi] = d;
  }
  P.h.nops = (int)sw.ops.size();
  P.h.ngacc = nacc;
  // offsets of each op's matrix and generator in the CTA's shared copy
  int soff = 0;
  for (int o = 0; o < P.h.nops; o++) {
    BOp& d = P.ops[o];
    const int dd = 1 << d.k;
    const int mc = d.kind == OPK_DIAG ? dd : d.kind == OPK_ANTIDIAG ? 2 : d.kind == OPK_SWAP ? 0 : dd * dd;
    const int gc = d.grad ? (d.kind == OPK_DIAG ? dd : dd * dd) : 0;
    d.soff = (uint16_t)soff;
    soff += mc + gc;
  }
  P.h.scoef = soff;

  // phases: consecutive ops whose moving qubits fit four register slots; tiles
  // of fewer than four qubits run every op in shared memory
  const bool reg_ok = sw.m >= kRegQ && sw.m - kRegQ <= 8;
  int nph = 0;
  auto add_phase = [&](PhaseKind kind, int first, int nops, uint32_t nd) {
    if (nph >= kMaxPhases) fail(SV_ERR_INVALID, "internal: too many phases");
    Phase& ph = P.ph[nph++];
    std::memset(&ph, 0, sizeof(ph));
    ph.kind = kind;
    ph.first = (uint8_t)first;
    ph.nops = (uint8_t)nops;
    if (kind != PH_REG) return;
    uint32_t rp = nd;
    if (__builtin_popcount(rp) < kRegQ && !(rp & 1u)) rp |= 1u;
    for (int q = sw.m - 1; q >= 0 && __builtin_popcount(rp) < kRegQ; q--) rp |= 1u << q;
    int slot_of[32], k2 = 0, nt = 0;
    for (int q = 0; q < sw.m; q++) {
      if ((rp >> q) & 1u) {
        slot_of[q] = k2;
        ph.rp[k2++] = (uint8_t)q;
      } else {
        slot_of[q] = -1;
        ph.tpos[nt++] = (uint8_t)q;
      }
    }
    ph.ntpos = (uint8_t)nt;
    ph.nrp = (uint8_t)k2;
    for (int o = first; o < first + nops; o++) {
      BOp& d = P.ops[o];
      for (int i = 0; i < d.k; i++)
        d.rs[i] = (d.pos[i] != 0xFF && slot_of[d.pos[i]] >= 0) ? (uint8_t)slot_of[d.pos[i]] : 0xFF;
      for (int q = 0; q < sw.m; q++) {
        if (!((d.lmask >> q) & 1u)) continue;
        const bool v = (d.lval >> q) & 1u;
        if (slot_of[q] >= 0) {
          d.rmask |= 1u << slot_of[q];
          if (v) d.rval |= 1u << slot_of[q];
        } else {
          d.tmask |= 1u << q;
          if (v) d.tval |= 1u << q;
        }
      }
    }
  };
  int cur_first = -1, cur_n = 0;
  uint32_t cur_need = 0;
  for (int o = 0; o < (int)sw.ops.size(); o++) {
    if (!reg_ok) {
      add_phase(PH_SMEM, o, 1, 0);
      continue;
    }
    if (cur_n && __builtin_popcount(cur_need | need[o]) <= kRegQ) {
      cur_need |= need[o];
      cur_n++;
    } else {
      if (cur_n) add_phase(PH_REG, cur_first, cur_n, cur_need);
      cur_first = o;
      cur_n = 1;
      cur_need = need[o];
    }
  }
  if (cur_n) add_phase(PH_REG, cur_first, cur_n, cur_need);
  P.h.nphases = nph;
}

// The batched programs of gates [g0, g1) of a template, one per pass over the
// batch: applied in order (forward), or un-applied in reverse order with
// their gradient terms (reverse); each(prog) is called for each in turn (prog
// is rewritten for the next).
template <typename R, typename F>
void segment_programs(const AdjTemplate& T, size_t g0, size_t g1, bool reverse, int n, int batch, int tile_q,
                      int low_q, BatchProgram<R>& prog, F&& each) {
  std::vector<int> order;
  std::vector<LOp> ops;
  if (!reverse) {
    for (size_t i = T.start[g0]; i < T.start[g1]; i++) {
      order.push_back((int)i);
      ops.push_back(T.ag[i].op);
    }
  } else {
    for (size_t i = T.start[g1]; i-- > T.start[g0];) {
      order.push_back((int)i);
      ops.push_back(T.ag[i].op);
    }
  }
  std::vector<Sweep> sws = schedule_sweeps(n, ops, tile_q, low_q, BatchProgram<R>::kPool / 2, 64);
  for (const Sweep& sw : sws) {
    fill_program<R>(T.ag, order, sw, n, batch, T.npg, reverse, prog);
    each(prog);
  }
}

// Tile width of the batched sweeps: 2^12 (complex64) or 2^11 (complex128)
// amplitudes: psi and lambda tiles fit shared memory twice over, and the
// register phases hold 16 amplitudes per thread with 256 threads.
// (Measured on the 20q HEA, batch 64: 12-qubit tiles 1511 gradient vectors/s,
// 11-qubit tiles with 128-thread CTAs 1498, 10-qubit 1337.)
int adjoint_tile_q(sv_dtype dtype) { return dtype == SV_C64 ? 12 : 11; }

// Every batched program of a call: forward segments of c gates, then (with
// reverse) the reverse segments; each(prog, rev).
template <typename R, typename F>
void all_programs(const AdjTemplate& T, size_t ng, int c, bool reverse, int n, sv_dtype dtype, int batch,
                  BatchProgram<R>& prog, F&& each) {
  const int tile_q = adjoint_tile_q(dtype), low_q = low_qubits_for(dtype);
  for (size_t a = 0; a < ng; a += c)
    segment_programs<R>(T, a, std::min(ng, a + c), false, n, batch, tile_q, low_q, prog,
                        [&](const BatchProgram<R>& P) { each(P, false); });
  if (!reverse) return;
  const int nseg = ng ? (int)((ng + c - 1) / c) : 0;
  for (int seg = nseg - 1; seg >= 0; seg--) {
    const size_t g0 = (size_t)seg * c, g1 = std::min(ng, g0 + c);
    segment_programs<R>(T, g0, g1, true, n, batch, tile_q, low_q, prog,
                        [&](const BatchProgram<R>& P) { each(P, true); });
  }
}

// Compiled batched kernels for a template: a template's calls are counted by
// its structure (gates without their angles, checkpoint interval, state size);
// on the call jit_mode() names (the second, or the first) every program of
// the call is written out and compiled, in parallel, and later launches find
// their kernels by program.  Returns whether launches should look them up.
std::mutex g_adj_jit_mu;
std::map<std::string, std::pair<int, int>> g_adj_jit;  // key -> (calls, parts compiled: 1 forward, 2 reverse)

template <typename R>
bool adjoint_jit(const AdjTemplate& T, const sv_gate* gates, size_t ng, int n, sv_dtype dtype, int batch, int c,
                 bool reverse) {
  const int mode = jit_mode();
  if (mode == 0) return false;
  std::string key;
  const int32_t hdr[3] = {n, (int32_t)dtype, c};  // the batch size changes no kernel
  key.append((const char*)hdr, sizeof(hdr));
  for (size_t i = 0; i < ng; i++) {
    sv_gate g = gates[i];
    g.matrix = nullptr;
    for (double& a : g.params) a = 0.0;
    key.append((const char*)&g, sizeof(g));
  }
  const int need = reverse ? 3 : 1;
  bool compile = false;
  {
    std::lock_guard<std::mutex> lk(g_adj_jit_mu);
    auto& e = g_adj_jit[key];
    e.first++;
    if (e.first < (mode == 2 ? 1 : 2)) return false;
    compile = (e.second & need) != need;
    e.second |= need;
  }
  if (compile) {
    std::vector<std::unique_ptr<BatchProgram<R>>> keep;
    std::vector<const BatchProgram<R>*> progs;
    std::vector<char> rev;
    std::unique_ptr<BatchProgram<R>> scratch(new BatchProgram<R>());
    all_programs<R>(T, ng, c, reverse, n, dtype, batch, *scratch, [&](const BatchProgram<R>& P, bool r) {
      keep.emplace_back(new BatchProgram<R>(P));
      progs.push_back(keep.back().get());
      rev.push_back(r ? 1 : 0);
    });
    jit_batch_prepare<R>(progs, rev);
  }
  return true;
}

template <typename R>
// With row_coeffs (host, batch x nterms) state b uses H_b = sum_j c_{b,j} P_j.
// With out_z (host, batch x (n + 1)) only the forward pass runs and
// <Z_q> of every state (then their sum) is returned.
// stored: how many of the segment-start states to keep (-1: all of them);
// the others are recomputed in the reverse pass by applying the gates again
// from the nearest kept state below (or |0..0>).
// dev: params, row_coeffs, out_grad, out_value and out_z are device arrays,
// the gate tables are built on the device and nothing is copied to the host
// (the call only enqueues work).  values_only: no reverse pass (out_grad
// unused).
void run_adjoint(int n, sv_dtype dtype, const sv_gate* gates, size_t ng, const double* params, int batch, int npar,
                 const sv_pauli_term* terms, size_t nterms, int ckpt, int stored, double* out_grad,
                 double* out_value, const double* row_coeffs, double* out_z, cudaStream_t stream, bool dev = false,
                 bool values_only = false) {
  const AdjTemplate tpl = lower_template(gates, ng);
  const std::vector<AGate>& ag = tpl.ag;
  const int npg = tpl.npg;

  // ---- per-state tables of the parameterised gates (double, then narrowed)
  const size_t N = 1ull << n;
  const size_t sbytes = sizeof(Cx<R>) * N * (size_t)batch;
  std::vector<Cx<R>> table(dev ? 0 : (size_t)std::max(npg, 1) * batch * kTableStride);
  std::vector<TableGate> tgates;
  std::vector<int> pslot;
  for (size_t i = 0; i < ag.size(); i++) {
    if (!ag[i].param) continue;
    tgates.push_back(TableGate{ag[i].rec.type, ag[i].slot});
    pslot.push_back(ag[i].slot);
    if (dev) continue;
    for (int b = 0; b < batch; b++) {
      std::vector<cplx> U = gate_matrix(ag[i].rec, params + (size_t)b * npar);
      Cx<R>* row = &table[((size_t)ag[i].pidx * batch + b) * kTableStride];
      int d = 1 << ag[i].rec.n_targets;
      if (ag[i].op.kind == OPK_DIAG)
        for (int r = 0; r < d; r++) row[r] = {(R)U[r * d + r].real(), (R)U[r * d + r].imag()};
      else
        for (int e = 0; e < d * d; e++) row[e] = {(R)U[e].real(), (R)U[e].imag()};
    }
  }

  // ---- device buffers (library-owned, per stream, grow-only)
  const int c = ckpt > 0 ? ckpt : (int)ng + 1;
  const int nck = ng > 0 ? (int)((ng - 1) / c) : 0;  // stored states after c, 2c, ... gates
  const int tile_q = adjoint_tile_q(dtype), low_q = low_qubits_for(dtype);
  const int m = std::min(n, tile_q);
  const int grid_x = batch_grid_x(n, m, batch);
  Cx<R>* psi = (Cx<R>*)scratch_buffer(stream, "adj_psi", sbytes);
  Cx<R>* lam = (Cx<R>*)scratch_buffer(stream, "adj_lam", sbytes);
  // boundaries j = 1..nck (the state after j*c gates); kept ones get a slot
  std::vector<int> slot_of(nck + 1, -1);
  int nkeep = stored < 0 ? nck : std::min(stored, nck);
  for (int i = 0; i < nkeep; i++) slot_of[(int)(((long long)(i + 1) * nck) / nkeep)] = i;  // evenly spaced
  Cx<R>* ck = nkeep ? (Cx<R>*)scratch_buffer(stream, "adj_ckpt", sbytes * nkeep) : nullptr;
  Cx<R>* dtab = (Cx<R>*)scratch_buffer(stream, "adj_table", sizeof(Cx<R>) * (size_t)std::max(npg, 1) * batch *
                                                                   kTableStride);
  double* gscr = (double*)scratch_buffer(stream, "adj_gscratch", sizeof(double) * (size_t)batch * std::max(npg, 1) * grid_x);
  double* gout = (double*)scratch_buffer(stream, "adj_gout", sizeof(double) * (size_t)batch * std::max(npg, 1));
  double* dots = (double*)scratch_buffer(stream, "adj_dot", sizeof(double) * batch_dot_scratch_doubles(batch));
  double* vout = (double*)scratch_buffer(stream, "adj_val", sizeof(double) * batch);
  int* dslot = nullptr;
  if (dev) {  // the gate list and slots go up (small); the matrices are built where the parameters are
    TableGate* dg = (TableGate*)scratch_buffer(stream, "adj_tgates", sizeof(TableGate) * std::max<size_t>(npg, 1));
    dslot = (int*)scratch_buffer(stream, "adj_pslot", sizeof(int) * std::max<size_t>(npg, 1));
    if (npg) {
      Pinned& pin = pinned_buffer(stream, "adj_tgates", sizeof(TableGate) * npg + sizeof(int) * npg);
      std::memcpy(pin.p, tgates.data(), sizeof(TableGate) * npg);
      std::memcpy((char*)pin.p + sizeof(TableGate) * npg, pslot.data(), sizeof(int) * npg);
      cuda_check(cudaMemcpyAsync(dg, pin.p, sizeof(TableGate) * npg, cudaMemcpyHostToDevice, stream), "gate list");
      cuda_check(cudaMemcpyAsync(dslot, (char*)pin.p + sizeof(TableGate) * npg, sizeof(int) * npg,
                                 cudaMemcpyHostToDevice, stream),
                 "slot list");
      cuda_check(cudaEventRecord(pin.ready, stream), "cudaEventRecord");
    }
    cuda_check(launch_build_tables<R>(params, npar, batch, dg, npg, dtab, stream), "gate tables");
  } else {
    cuda_check(cudaMemcpyAsync(dtab, table.data(), table.size() * sizeof(Cx<R>), cudaMemcpyHostToDevice, stream),
               "table upload");
  }

  std::unique_ptr<BatchProgram<R>> prog(new BatchProgram<R>());
  const double sweep_bytes_f = 2.0 * (double)sbytes, sweep_bytes_r = 4.0 * (double)sbytes;
  // the programs' compiled kernels, from the call jit_mode() names on
  const bool jit = adjoint_jit<R>(tpl, gates, ng, n, dtype, batch, c, !out_z && !values_only);
  auto sweep = [&](const BatchProgram<R>& P, bool rev) {
    const JitKernel* k = jit ? jit_batch_lookup<R>(P, rev) : nullptr;
    Prof pr(stream, rev ? (k ? "batch_sweep_rev_jit" : "batch_sweep_rev") : (k ? "batch_sweep_fwd_jit" : "batch_sweep_fwd"),
            rev ? sweep_bytes_r : sweep_bytes_f);
    cuda_check(launch_batch_sweep<R>(psi, rev ? lam : nullptr, dtab, gscr, grid_x, P, rev, stream, k),
               rev ? "reverse sweep" : "forward sweep");
    pr.done();
  };

  // ---- forward over gates [g0, g1) in segments of c, keeping the chosen
  // segment-start states when `keep`
  auto forward = [&](size_t g0, size_t g1, bool keep) {
    for (size_t a = g0; a < g1; a += c) {
      const size_t b = std::min(g1, a + c);
      segment_programs<R>(tpl, a, b, false, n, batch, tile_q, low_q, *prog,
                          [&](const BatchProgram<R>& P) { sweep(P, false); });
      const int j = (int)(b / c);  // boundary reached (state after j*c gates)
      if (keep && b % c == 0 && j >= 1 && j <= nck && slot_of[j] >= 0)
        cuda_check(cudaMemcpyAsync(ck + (size_t)slot_of[j] * N * batch, psi, sbytes, cudaMemcpyDeviceToDevice, stream),
                   "checkpoint store");
    }
  };
  cuda_check(launch_batch_init<R>(psi, n, batch, stream), "batch init");
  forward(0, ng, true);

  // ---- forward-only: <Z_q> of every state
  if (out_z) {
    const size_t zn = (size_t)n + 1;
    double* zscr = (double*)scratch_buffer(stream, "adj_zscratch", sizeof(double) * expect_z_all_scratch_doubles(n));
    double* zdev = dev ? out_z : (double*)scratch_buffer(stream, "adj_zout", sizeof(double) * zn * batch);
    for (int b = 0; b < batch; b++)
      cuda_check(launch_expect_z_all<R>(psi + (size_t)b * N, n, zscr, expect_z_all_scratch_doubles(n),
                                        zdev + (size_t)b * zn, stream),
                 "per-state <Z>");
    if (dev) return;
    cuda_check(cudaMemcpyAsync(out_z, zdev, sizeof(double) * zn * batch, cudaMemcpyDeviceToHost, stream),
               "<Z> copy");
    cuda_check(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    return;
  }

  // ---- lambda = H psi (tiles that hold whole X-masks); f = Re <psi|lambda>
  {
    const double* rowc = nullptr;
    if (row_coeffs && dev) {
      rowc = row_coeffs;
    } else if (row_coeffs) {
      double* up = (double*)scratch_buffer(stream, "adj_rowc", sizeof(double) * nterms * batch);
      cuda_check(cudaMemcpyAsync(up, row_coeffs, sizeof(double) * nterms * batch, cudaMemcpyHostToDevice, stream),
                 "row coefficients upload");
      rowc = up;
    }
    Prof pr(stream, "pauli_accum", 2.0 * (double)sbytes);
    const cudaError_t e = launch_pauli_tiles<R>(psi, lam, n, batch, terms, (int)nterms, false, rowc, stream);
    if (e == cudaErrorNotSupported)
      fail(SV_ERR_UNSUPPORTED, "per-state coefficients need every X-mask to fit one tile of " +
                                   std::to_string(dtype == SV_C64 ? 13 : 12) + " qubits (with the lowest ones)");
    cuda_check(e, "H psi");
    pr.done();
    cuda_check(launch_batch_dot<R>(psi, lam, n, batch, dots, vout, stream), "value");
  }
  if (values_only) {
    if (dev) {
      cuda_check(cudaMemcpyAsync(out_value, vout, sizeof(double) * batch, cudaMemcpyDeviceToDevice, stream),
                 "value copy");
    } else {
      cuda_check(cudaMemcpyAsync(out_value, vout, sizeof(double) * batch, cudaMemcpyDeviceToHost, stream),
                 "value copy");
      cuda_check(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    }
    return;
  }

  // ---- reverse, segment by segment, re-anchoring psi at checkpoints
  int nseg = ng ? (int)((ng + c - 1) / c) : 0;
  for (int seg = nseg - 1; seg >= 0; seg--) {
    size_t g0 = (size_t)seg * c, g1 = std::min(ng, g0 + c);
    segment_programs<R>(tpl, g0, g1, true, n, batch, tile_q, low_q, *prog,
                        [&](const BatchProgram<R>& P) { sweep(P, true); });
    if (seg >= 1 && seg <= nck) {  // psi is now psi after seg*c gates: re-anchor it
      if (slot_of[seg] >= 0) {
        cuda_check(cudaMemcpyAsync(psi, ck + (size_t)slot_of[seg] * N * batch, sbytes, cudaMemcpyDeviceToDevice,
                                   stream),
                   "checkpoint load");
      } else {  // recompute from the nearest kept state below, or from |0..0>
        int i = seg - 1;
        while (i >= 1 && slot_of[i] < 0) i--;
        if (i >= 1)
          cuda_check(cudaMemcpyAsync(psi, ck + (size_t)slot_of[i] * N * batch, sbytes, cudaMemcpyDeviceToDevice,
                                     stream),
                     "checkpoint load");
        else
          cuda_check(launch_batch_init<R>(psi, n, batch, stream), "batch init");
        forward((size_t)(i >= 1 ? i : 0) * c, (size_t)seg * c, false);
      }
    }
  }
  if (npg) cuda_check(launch_grad_finish(gscr, batch, npg, grid_x, gout, stream), "gradient reduce");
  if (dev) {  // slots shared by several gates add up, on the device
    if (npg) {
      cuda_check(launch_scatter_grad(gout, batch, npg, dslot, npar, out_grad, stream), "gradient scatter");
    } else if (npar) {
      cuda_check(cudaMemsetAsync(out_grad, 0, sizeof(double) * (size_t)batch * npar, stream), "gradient clear");
    }
    cuda_check(cudaMemcpyAsync(out_value, vout, sizeof(double) * batch, cudaMemcpyDeviceToDevice, stream),
               "value copy");
    return;
  }

  // ---- results to the host; slots shared by several gates add up
  std::vector<double> gh((size_t)batch * std::max(npg, 1), 0.0);
  if (npg)
    cuda_check(cudaMemcpyAsync(gh.data(), gout, sizeof(double) * gh.size(), cudaMemcpyDeviceToHost, stream),
               "gradient copy");
  cuda_check(cudaMemcpyAsync(out_value, vout, sizeof(double) * batch, cudaMemcpyDeviceToHost, stream), "value copy");
  cuda_check(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
  std::fill(out_grad, out_grad + (size_t)batch * npar, 0.0);
  for (size_t i = 0; i < ag.size(); i++) {
    if (!ag[i].param) continue;
    for (int b = 0; b < batch; b++) out_grad[(size_t)b * npar + ag[i].slot] += gh[(size_t)b * npg + ag[i].pidx];
  }
}

}  // namespace
}  // namespace sv

using namespace sv;

namespace {

void check_adjoint_args(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates, const double* params,
                        int batch, int n_params, int checkpoint_every) {
  if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_INVALID, "unknown dtype");
  if (n_qubits < 1 || n_qubits > 30) fail(SV_ERR_INVALID, "n_qubits must be in 1..30 for the adjoint");
  if (batch < 1 || batch > 65535) fail(SV_ERR_INVALID, "batch must be in 1..65535");
  if (n_params < 0) fail(SV_ERR_INVALID, "n_params must be >= 0");
  if (n_params > 0 && !params) fail(SV_ERR_INVALID, "params is NULL");
  if (checkpoint_every < 0) fail(SV_ERR_INVALID, "checkpoint_every must be >= 0");
  validate_gates(n_qubits, gates, n_gates, (size_t)n_params);
  for (int b = 0; b < batch; b++)
    for (int p = 0; p < n_params; p++)
      if (!std::isfinite(params[(size_t)b * n_params + p])) fail(SV_ERR_INVALID, "a parameter is not finite");
}

void check_terms(int n_qubits, const sv_pauli_term* terms, size_t n_terms) {
  if (n_terms < 1 || n_terms > 4096 || !terms) fail(SV_ERR_INVALID, "n_terms must be in 1..4096");
  const uint64_t all = (1ull << n_qubits) - 1ull;
  for (size_t j = 0; j < n_terms; j++)
    if ((terms[j].x_mask | terms[j].z_mask) & ~all)
      fail(SV_ERR_INVALID, "term " + std::to_string(j) + " names a qubit beyond n_qubits");
}

void adjoint_dispatch(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates, const double* params,
                      int batch, int n_params, const sv_pauli_term* terms, size_t n_terms, int checkpoint_every,
                      double* out_grad, double* out_value, const double* row_coeffs, double* out_z, void* stream,
                      int stored = -1, bool dev = false, bool values_only = false) {
  static double dummy_grad;
  double* og = n_params > 0 && out_grad ? out_grad : &dummy_grad;
  if (dtype == SV_C64)
    run_adjoint<float>(n_qubits, dtype, gates, n_gates, params, batch, n_params, terms, n_terms, checkpoint_every,
                       stored, og, out_value, row_coeffs, out_z, (cudaStream_t)stream, dev, values_only);
  else
    run_adjoint<double>(n_qubits, dtype, gates, n_gates, params, batch, n_params, terms, n_terms, checkpoint_every,
                        stored, og, out_value, row_coeffs, out_z, (cudaStream_t)stream, dev, values_only);
}

// As check_adjoint_args for device-resident parameters (their values are not
// read on the host).
void check_adjoint_args_dev(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates, const double* params,
                            int batch, int n_params, int checkpoint_every) {
  if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_INVALID, "unknown dtype");
  if (n_qubits < 1 || n_qubits > 30) fail(SV_ERR_INVALID, "n_qubits must be in 1..30 for the adjoint");
  if (batch < 1 || batch > 65535) fail(SV_ERR_INVALID, "batch must be in 1..65535");
  if (n_params < 0) fail(SV_ERR_INVALID, "n_params must be >= 0");
  if (checkpoint_every < 0) fail(SV_ERR_INVALID, "checkpoint_every must be >= 0");
  if (n_params > 0) check_device_buffer(params, sizeof(double) * (size_t)batch * n_params, "params");
  validate_gates(n_qubits, gates, n_gates, (size_t)n_params);
}

}  // namespace

namespace {

template <typename R>
void check_adjoint_kernels(const AdjTemplate& T, size_t ng, int c, int n, sv_dtype dtype, bool compile, int arch,
                           int* n_sources, int* n_compiled, std::string* err, std::string* src) {
  std::vector<std::unique_ptr<BatchProgram<R>>> keep;
  std::vector<const BatchProgram<R>*> progs;
  std::vector<char> rev;
  std::unique_ptr<BatchProgram<R>> scratch(new BatchProgram<R>());
  all_programs<R>(T, ng, c, true, n, dtype, 1, *scratch, [&](const BatchProgram<R>& P, bool r) {
    keep.emplace_back(new BatchProgram<R>(P));
    progs.push_back(keep.back().get());
    rev.push_back(r ? 1 : 0);
  });
  jit_check_batch<R>(progs, rev, compile, arch, n_sources, n_compiled, err, src);
}

}  // namespace

extern "C" sv_status sv_jit_check_adjoint(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                                          int n_params, int checkpoint_every, int compile, int arch, int* n_sources,
                                          int* n_compiled, char* text, size_t text_cap) {
  return guarded([&] {
    if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_INVALID, "unknown dtype");
    if (n_qubits < 1 || n_qubits > 30) fail(SV_ERR_INVALID, "n_qubits must be in 1..30 for the adjoint");
    if (n_params < 0 || checkpoint_every < 0) fail(SV_ERR_INVALID, "n_params and checkpoint_every must be >= 0");
    if (!n_sources || !n_compiled) fail(SV_ERR_INVALID, "NULL argument");
    if (compile && (arch < 100 || arch > 200)) fail(SV_ERR_INVALID, "arch must be a compute capability such as 103");
    if (compile && !jit_available(nullptr)) fail(SV_ERR_UNSUPPORTED, "the run-time compiler is not available");
    validate_gates(n_qubits, gates, n_gates, (size_t)n_params);
    const AdjTemplate T = lower_template(gates, n_gates);
    const int c = checkpoint_every > 0 ? checkpoint_every : (int)n_gates + 1;
    std::string err, src;
    if (dtype == SV_C64)
      check_adjoint_kernels<float>(T, n_gates, c, n_qubits, dtype, compile != 0, arch, n_sources, n_compiled, &err,
                                   &src);
    else
      check_adjoint_kernels<double>(T, n_gates, c, n_qubits, dtype, compile != 0, arch, n_sources, n_compiled, &err,
                                    &src);
    if (text && text_cap) {
      const std::string& m = err.empty() ? src : err;
      const size_t k = std::min(m.size(), text_cap - 1);
      std::memcpy(text, m.data(), k);
      text[k] = '\0';
    }
  });
}

extern "C" sv_status sv_adjoint_grad(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                                     const double* params, int batch, int n_params, const sv_pauli_term* terms,
                                     size_t n_terms, int checkpoint_every, double* out_grad, double* out_value,
                                     void* stream) {
  return guarded([&] {
    check_adjoint_args(n_qubits, dtype, gates, n_gates, params, batch, n_params, checkpoint_every);
    check_terms(n_qubits, terms, n_terms);
    if (!out_grad && n_params > 0) fail(SV_ERR_INVALID, "out_grad is NULL");
    if (!out_value) fail(SV_ERR_INVALID, "out_value is NULL");
    adjoint_dispatch(n_qubits, dtype, gates, n_gates, params, batch, n_params, terms, n_terms, checkpoint_every,
                     out_grad, out_value, nullptr, nullptr, stream);
  });
}

extern "C" sv_status sv_adjoint_grad_rows(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                                          const double* params, int batch, int n_params, const sv_pauli_term* terms,
                                          size_t n_terms, const double* row_coeffs, int checkpoint_every,
                                          double* out_grad, double* out_value, void* stream) {
  return guarded([&] {
    check_adjoint_args(n_qubits, dtype, gates, n_gates, params, batch, n_params, checkpoint_every);
    check_terms(n_qubits, terms, n_terms);
    if (!row_coeffs) fail(SV_ERR_INVALID, "row_coeffs is NULL");
    for (size_t i = 0; i < (size_t)batch * n_terms; i++)
      if (!std::isfinite(row_coeffs[i])) fail(SV_ERR_INVALID, "a coefficient is not finite");
    if (!out_grad && n_params > 0) fail(SV_ERR_INVALID, "out_grad is NULL");
    if (!out_value) fail(SV_ERR_INVALID, "out_value is NULL");
    adjoint_dispatch(n_qubits, dtype, gates, n_gates, params, batch, n_params, terms, n_terms, checkpoint_every,
                     out_grad, out_value, row_coeffs, nullptr, stream);
  });
}

extern "C" sv_status sv_batch_expect_z(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                                       const double* params, int batch, int n_params, double* out_z, void* stream) {
  return guarded([&] {
    check_adjoint_args(n_qubits, dtype, gates, n_gates, params, batch, n_params, 0);
    if (!out_z) fail(SV_ERR_INVALID, "out_z is NULL");
    static const sv_pauli_term z0 = {0, 1, 1.0};  // unused: forward only
    double value_unused = 0.0;
    adjoint_dispatch(n_qubits, dtype, gates, n_gates, params, batch, n_params, &z0, 1, 0, nullptr, &value_unused,
                     nullptr, out_z, stream);
  });
}

extern "C" sv_status sv_adjoint_grad_ex(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                                        const double* params, int batch, int n_params, const sv_pauli_term* terms,
                                        size_t n_terms, const sv_adjoint_opts* opts, double* out_grad,
                                        double* out_value, void* stream) {
  return guarded([&] {
    if (!opts) fail(SV_ERR_INVALID, "opts is NULL");
    check_adjoint_args(n_qubits, dtype, gates, n_gates, params, batch, n_params, opts->checkpoint_every);
    check_terms(n_qubits, terms, n_terms);
    if (!out_grad && n_params > 0) fail(SV_ERR_INVALID, "out_grad is NULL");
    if (!out_value) fail(SV_ERR_INVALID, "out_value is NULL");
    if (opts->stored_states < -1) fail(SV_ERR_INVALID, "stored_states must be >= -1");
    if (!(opts->memory_budget_bytes >= 0.0)) fail(SV_ERR_INVALID, "memory_budget_bytes must be >= 0");
    int stored = opts->stored_states;
    if (opts->memory_budget_bytes > 0.0) {  // automatic placement: as many states as the budget holds
      const double state_bytes = (double)(dtype == SV_C64 ? 8 : 16) * (double)(1ull << n_qubits) * (double)batch;
      const double fit = std::floor(opts->memory_budget_bytes / state_bytes);
      stored = fit > 1e9 ? -1 : (int)fit;
    }
    adjoint_dispatch(n_qubits, dtype, gates, n_gates, params, batch, n_params, terms, n_terms,
                     opts->checkpoint_every, out_grad, out_value, nullptr, nullptr, stream, stored);
  });
}

extern "C" sv_status sv_adjoint_grad_device(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                                            const double* params, int batch, int n_params,
                                            const sv_pauli_term* terms, size_t n_terms, const double* row_coeffs,
                                            int checkpoint_every, double* out_grad, double* out_value,
                                            void* stream) {
  return guarded([&] {
    check_adjoint_args_dev(n_qubits, dtype, gates, n_gates, params, batch, n_params, checkpoint_every);
    check_terms(n_qubits, terms, n_terms);
    if (row_coeffs) check_device_buffer(row_coeffs, sizeof(double) * (size_t)batch * n_terms, "row_coeffs");
    if (out_grad && n_params > 0) check_device_buffer(out_grad, sizeof(double) * (size_t)batch * n_params, "out_grad");
    check_device_buffer(out_value, sizeof(double) * (size_t)batch, "out_value");
    adjoint_dispatch(n_qubits, dtype, gates, n_gates, params, batch, n_params, terms, n_terms, checkpoint_every,
                     out_grad, out_value, row_coeffs, nullptr, stream, -1, true, out_grad == nullptr);
  });
}

extern "C" sv_status sv_batch_expect_z_device(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                                              const double* params, int batch, int n_params, double* out_z,
                                              void* stream) {
  return guarded([&] {
    check_adjoint_args_dev(n_qubits, dtype, gates, n_gates, params, batch, n_params, 0);
    check_device_buffer(out_z, sizeof(double) * (size_t)batch * (n_qubits + 1), "out_z");
    static const sv_pauli_term z0 = {0, 1, 1.0};  // unused: forward only
    adjoint_dispatch(n_qubits, dtype, gates, n_gates, params, batch, n_params, &z0, 1, 0, nullptr, nullptr, nullptr,
                     out_z, stream, -1, true);
  });
}
