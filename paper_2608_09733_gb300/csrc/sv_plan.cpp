// sv_plan.cpp -- host side of the gate-application path.
//
//  * validation of gate records at the boundary (Sec. 3.3: unsupported or
//    unbound inputs raise instead of being approximated);
//  * lowering of each gate to its matrix in double precision (Sec. 3.3 and
//    Sec. 5.2: build at the widest precision, narrow at the device boundary);
//  * classification into the fast paths the paper names (Sec. 5.3 real vs
//    complex gates; Sec. 9.2 diagonal and permutation paths);
//  * the paper's fusion (Sec. 4.3 `fuse`, Sec. 9.2): consecutive gates are
//    joined, without reordering, while their qubits fit k;
//  * the tile scheduler: packs consecutive operations whose non-diagonal
//    qubits fit one shared-memory tile into a single pass over HBM.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>

#include "sv_internal.h"

namespace sv {

namespace {

const int kTargetsOf[SV_GATE_COUNT_] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1,  // I..SX
                                        1, 1, 1, 1, 1, 1,              // RX..U3
                                        2, 2, 2, 2,                    // SWAP, RXX, RYY, RZZ
                                        -1,                            // UNITARY
                                        2, 4};                         // EXC1, EXC2
const int kAnglesOf[SV_GATE_COUNT_] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 2, 3, 0, 1, 1, 1, 0, 1, 1};

uint64_t gate_qubit_mask(const sv_gate& g) {
  uint64_t m = 0;
  for (int i = 0; i < g.n_targets; i++) m |= 1ull << g.targets[i];
  for (int i = 0; i < g.n_controls; i++) m |= 1ull << g.controls[i];
  return m;
}

int popc(uint64_t x) { return __builtin_popcountll(x); }

}  // namespace

#ifndef SV_C64_TILE_Q
#define SV_C64_TILE_Q 13  // 64 KiB tiles, five register qubits per phase
#endif
#ifndef SV_C64_SMALL_TILE_MIN_N
#define SV_C64_SMALL_TILE_MIN_N 26
#endif
#ifndef SV_C64_TMA_MIN_N
#define SV_C64_TMA_MIN_N 21  // 2^9 tiles of 12 qubits: the TMA pass
#endif
// complex64 states of 2^26 amplitudes and more run 12-qubit tiles: four
// 128-thread CTAs per SM instead of two 256-thread ones hide the tile copies
// and barriers better (measured 6-8 % less time per step at 26-30 qubits on
// layered circuits, despite about 15 % more passes).  States of 21 to 25
// qubits take 12-qubit tiles too when their passes can run compiled (the
// compiled kernels are on and NVRTC is present): the TMA pass on 12-qubit
// tiles with compiled programs beats the interpreted pass on 13-qubit tiles
// by 1.27x at 22 and 24 qubits and 1.5x at 25 on layered circuits, with
// 10-15 % more passes, and interpreted (a program structure's first run) it
// is no slower.  The serving circuits' CNOT ladders take 14-28 % more passes
// on 12-qubit tiles at 21-25 qubits, which their compiled passes (1.5-1.8x
// faster) more than repay once a structure has run twice.  Smaller states
// keep the wider tile.
int tile_qubits_for(sv_dtype dtype, int n) {
  if (dtype != SV_C64) return 11;
  if (n >= SV_C64_SMALL_TILE_MIN_N) return SV_C64_TILE_Q - 1;
  if (n >= SV_C64_TMA_MIN_N && jit_mode() != 0 && jit_available(nullptr)) return SV_C64_TILE_Q - 1;
  return SV_C64_TILE_Q;
}
#ifndef SV_RQ5_MIN_M
#define SV_RQ5_MIN_M 12  // tiles of at least this many qubits use five register qubits
#endif
int reg_qubits_for(int m) { return m >= SV_RQ5_MIN_M ? 5 : kRegQ; }
int low_qubits_for(sv_dtype dtype) { return dtype == SV_C64 ? 5 : 4; }     // 256-byte runs

void validate_gates(int n, const sv_gate* gates, size_t n_gates, size_t n_param_values) {
  if (n_gates && !gates) fail(SV_ERR_INVALID, "gates is NULL");
  for (size_t gi = 0; gi < n_gates; gi++) {
    const sv_gate& g = gates[gi];
    std::string at = "gate " + std::to_string(gi) + ": ";
    if (g.type < 0 || g.type >= SV_GATE_COUNT_) fail(SV_ERR_INVALID, at + "unknown gate type");
    int want = kTargetsOf[g.type];
    if (want > 0 && g.n_targets != want) fail(SV_ERR_INVALID, at + "wrong number of targets for its family");
    if (g.n_targets < 1 || g.n_targets > SV_MAX_TARGETS) fail(SV_ERR_INVALID, at + "n_targets out of range");
    if (g.n_controls < 0 || g.n_controls > SV_MAX_CONTROLS) fail(SV_ERR_INVALID, at + "n_controls out of range");
    uint64_t seen = 0;
    for (int i = 0; i < g.n_targets + g.n_controls; i++) {
      int q = i < g.n_targets ? g.targets[i] : g.controls[i - g.n_targets];
      if (q < 0 || q >= n) fail(SV_ERR_INVALID, at + "qubit " + std::to_string(q) + " out of range");
      if (seen & (1ull << q)) fail(SV_ERR_INVALID, at + "qubit " + std::to_string(q) + " repeated");
      seen |= 1ull << q;
    }
    if (g.n_controls < 32 && (g.control_zero_mask >> g.n_controls) != 0)
      fail(SV_ERR_INVALID, at + "control_zero_mask has bits beyond n_controls");
    for (int i = 0; i < kAnglesOf[g.type]; i++) {
      int s = g.param_slot[i];
      if (s < -1) fail(SV_ERR_INVALID, at + "negative parameter slot");
      if (s >= 0 && (size_t)s >= n_param_values)
        fail(SV_ERR_UNBOUND_PARAM, at + "parameter slot " + std::to_string(s) + " is unbound");
      double v = s >= 0 ? 0.0 : g.params[i];
      if (!std::isfinite(v)) fail(SV_ERR_INVALID, at + "angle is not finite");
    }
    if (g.type == SV_GATE_UNITARY) {
      if (!g.matrix) fail(SV_ERR_INVALID, at + "unitary gate without a matrix");
      int d = 1 << g.n_targets;
      // U^dagger U = I within 1e-6 (a user matrix that is not unitary is rejected)
      double worst = 0.0;
      for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) {
          cplx acc = 0.0;
          for (int k = 0; k < d; k++) {
            cplx a(g.matrix[2 * (k * d + r)], -g.matrix[2 * (k * d + r) + 1]);
            cplx b(g.matrix[2 * (k * d + c)], g.matrix[2 * (k * d + c) + 1]);
            acc += a * b;
          }
          worst = std::max(worst, std::abs(acc - (r == c ? 1.0 : 0.0)));
        }
      if (!(worst < 1e-6)) fail(SV_ERR_INVALID, at + "matrix is not unitary");
    }
  }
}

// The matrix of a gate (without its controls), from the definitions of the
// gate table (Sec. 4.2) and R_P(theta) = exp(-i theta P / 2) (Sec. 9.1).
std::vector<cplx> gate_matrix(const sv_gate& g, const double* pv) {
  auto ang = [&](int i) { return g.param_slot[i] >= 0 ? pv[g.param_slot[i]] : g.params[i]; };
  const cplx j(0.0, 1.0);
  const double h = 1.0 / std::sqrt(2.0);
  switch (g.type) {
    case SV_GATE_I: return {1.0, 0.0, 0.0, 1.0};
    case SV_GATE_X: return {0.0, 1.0, 1.0, 0.0};
    case SV_GATE_Y: return {0.0, -j, j, 0.0};
    case SV_GATE_Z: return {1.0, 0.0, 0.0, -1.0};
    case SV_GATE_H: return {h, h, h, -h};
    case SV_GATE_S: return {1.0, 0.0, 0.0, j};
    case SV_GATE_SDG: return {1.0, 0.0, 0.0, -j};
    case SV_GATE_T: return {1.0, 0.0, 0.0, std::polar(1.0, M_PI / 4.0)};
    case SV_GATE_TDG: return {1.0, 0.0, 0.0, std::polar(1.0, -M_PI / 4.0)};
    case SV_GATE_SX: return {0.5 * (1.0 + j), 0.5 * (1.0 - j), 0.5 * (1.0 - j), 0.5 * (1.0 + j)};
    case SV_GATE_RX: {
      double c = std::cos(0.5 * ang(0)), s = std::sin(0.5 * ang(0));
      return {c, -j * s, -j * s, c};
    }
    case SV_GATE_RY: {
      double c = std::cos(0.5 * ang(0)), s = std::sin(0.5 * ang(0));
      return {c, -s, s, c};
    }
    case SV_GATE_RZ: return {std::polar(1.0, -0.5 * ang(0)), 0.0, 0.0, std::polar(1.0, 0.5 * ang(0))};
    case SV_GATE_P: return {1.0, 0.0, 0.0, std::polar(1.0, ang(0))};
    case SV_GATE_U2:
    case SV_GATE_U3: {
      double th = g.type == SV_GATE_U2 ? M_PI / 2.0 : ang(0);
      double ph = g.type == SV_GATE_U2 ? ang(0) : ang(1);
      double la = g.type == SV_GATE_U2 ? ang(1) : ang(2);
      double c = std::cos(0.5 * th), s = std::sin(0.5 * th);
      return {c, -std::polar(s, la), std::polar(s, ph), std::polar(c, ph + la)};
    }
    case SV_GATE_SWAP: {
      std::vector<cplx> m(16, 0.0);
      m[0] = m[15] = 1.0;
      m[1 * 4 + 2] = m[2 * 4 + 1] = 1.0;
      return m;
    }
    case SV_GATE_RXX:
    case SV_GATE_RYY: {
      // cos(t/2) I - i sin(t/2) P(x)P; XX and YY are anti-diagonal, YY has
      // -1 on its outer anti-diagonal corners and +1 on the inner ones.
      double c = std::cos(0.5 * ang(0)), s = std::sin(0.5 * ang(0));
      double outer = g.type == SV_GATE_RXX ? 1.0 : -1.0;
      std::vector<cplx> m(16, 0.0);
      for (int r = 0; r < 4; r++) m[r * 4 + r] = c;
      m[0 * 4 + 3] = m[3 * 4 + 0] = -j * s * outer;
      m[1 * 4 + 2] = m[2 * 4 + 1] = -j * s;
      return m;
    }
    case SV_GATE_RZZ: {
      // Z(x)Z = diag(1, -1, -1, 1)
      cplx a = std::polar(1.0, -0.5 * ang(0)), b = std::polar(1.0, 0.5 * ang(0));
      std::vector<cplx> m(16, 0.0);
      m[0] = a; m[5] = b; m[10] = b; m[15] = a;
      return m;
    }
    case SV_GATE_UNITARY: {
      int d = 1 << g.n_targets;
      std::vector<cplx> m(d * d);
      for (int i = 0; i < d * d; i++) m[i] = cplx(g.matrix[2 * i], g.matrix[2 * i + 1]);
      return m;
    }
    case SV_GATE_EXC1:
    case SV_GATE_EXC2: {
      // identity except the rotation [[c, -s], [s, c]] on the two states that
      // exchange the excitation: indices (1, 2) of 4, or (3, 12) of 16
      const int d = g.type == SV_GATE_EXC1 ? 4 : 16, a = g.type == SV_GATE_EXC1 ? 1 : 3,
                b = g.type == SV_GATE_EXC1 ? 2 : 12;
      const double c = std::cos(0.5 * ang(0)), s = std::sin(0.5 * ang(0));
      std::vector<cplx> m(d * d, 0.0);
      for (int r = 0; r < d; r++) m[r * d + r] = 1.0;
      m[a * d + a] = c;
      m[a * d + b] = -s;
      m[b * d + a] = s;
      m[b * d + b] = c;
      return m;
    }
    default: fail(SV_ERR_INVALID, "unknown gate type");
  }
}

void classify(LOp& op) {
  const int d = 1 << op.k;
  const std::vector<cplx>& m = op.m;
  op.touch = 0;
  for (int i = 0; i < op.k; i++) op.touch |= 1ull << op.q[i];
  for (int i = 0; i < op.nc; i++) op.touch |= 1ull << op.c[i];
  uint64_t tq = 0;
  for (int i = 0; i < op.k; i++) tq |= 1ull << op.q[i];

  bool diag = true, real = true;
  for (int r = 0; r < d; r++)
    for (int c = 0; c < d; c++) {
      const cplx& v = m[r * d + c];
      if (r != c && v != 0.0) diag = false;
      if (v.imag() != 0.0) real = false;
    }
  if (diag) {
    std::vector<cplx> dd(d);
    for (int r = 0; r < d; r++) dd[r] = m[r * d + r];
    op.kind = OPK_DIAG;
    op.m = dd;
    op.need = 0;  // a diagonal never moves amplitudes: any tile can apply it
    return;
  }
  if (op.k == 1 && m[0] == 0.0 && m[3] == 0.0) {
    op.kind = OPK_ANTIDIAG;
    op.m = {m[1], m[2]};
    op.need = tq;
    return;
  }
  if (op.k == 2) {
    bool sw = true;
    for (int r = 0; r < 4; r++)
      for (int c = 0; c < 4; c++) {
        int want_c = (r == 1) ? 2 : (r == 2) ? 1 : r;
        if (m[r * 4 + c] != (c == want_c ? 1.0 : 0.0)) sw = false;
      }
    if (sw) {
      op.kind = OPK_SWAP;
      op.m.clear();
      op.need = tq;
      return;
    }
  }
  op.kind = (real && op.k <= 2) ? OPK_REAL : OPK_DENSE;
  op.need = tq;
}

LOp lower_gate(const sv_gate& g, const double* pv, int index) {
  LOp op;
  op.k = g.n_targets;
  for (int i = 0; i < op.k; i++) op.q[i] = g.targets[i];
  op.nc = g.n_controls;
  for (int i = 0; i < op.nc; i++) {
    op.c[i] = g.controls[i];
    op.cs[i] = ((g.control_zero_mask >> i) & 1u) ? 0 : 1;
  }
  op.m = gate_matrix(g, pv);
  op.first_gate = index;
  classify(op);
  return op;
}

// Applies gate g, re-indexed onto the block's local qubits, to a vector of
// 2^nb amplitudes (used to build a fused block's matrix column by column).
static void apply_local(std::vector<cplx>& v, int nb, const sv_gate& g, const std::vector<cplx>& U,
                        const int* local_of) {
  int k = g.n_targets, d = 1 << k;
  int t[5];
  for (int i = 0; i < k; i++) t[i] = local_of[g.targets[i]];
  uint64_t cmask = 0, cval = 0;
  for (int i = 0; i < g.n_controls; i++) {
    int lq = local_of[g.controls[i]];
    cmask |= 1ull << lq;
    if (!((g.control_zero_mask >> i) & 1u)) cval |= 1ull << lq;
  }
  uint64_t tmask = 0;
  for (int i = 0; i < k; i++) tmask |= 1ull << t[i];
  cplx in[32];  // k <= 5
  for (uint64_t b = 0; b < (1ull << nb); b++) {
    if (b & tmask) continue;  // enumerate group bases (target bits clear)
    if ((b & cmask) != cval) continue;
    for (int jj = 0; jj < d; jj++) {
      uint64_t idx = b;
      for (int i = 0; i < k; i++)
        if ((jj >> i) & 1) idx |= 1ull << t[i];
      in[jj] = v[idx];
    }
    for (int r = 0; r < d; r++) {
      cplx acc = 0.0;
      for (int c = 0; c < d; c++) acc += U[r * d + c] * in[c];
      uint64_t idx = b;
      for (int i = 0; i < k; i++)
        if ((r >> i) & 1) idx |= 1ull << t[i];
      v[idx] = acc;
    }
  }
}

// Cost per amplitude of one operation inside a pass, in the kernel's terms:
// the multiply-adds of its complex matrix-vector product as real flops, plus
// the overhead of the path it takes.  One- and two-qubit ops run on register
// groups (a few integer ops of overhead); wider dense blocks and diagonals run
// group by group in shared memory (an address computation and a shared-memory
// round trip per amplitude).  A sign flip (Z, CZ) and a bit flip (X, CNOT)
// cost almost nothing.
double op_cost(const LOp& op) {
  const bool wide = op.k >= 3;
  switch (op.kind) {
    case OPK_DENSE: return 8.0 * (1 << op.k) + (wide ? 40.0 : 2.0);
    case OPK_REAL: return 4.0 * (1 << op.k) + (wide ? 40.0 : 2.0);
    case OPK_DIAG: {
      const int d = 1 << op.k;
      bool sign = true;
      for (int r = 0; r < d && r < (int)op.m.size(); r++)
        if (op.m[r] != (r == d - 1 ? cplx(-1.0) : cplx(1.0))) sign = false;
      if (sign) return 1.0;
      return wide ? 60.0 : 10.0;
    }
    case OPK_ANTIDIAG: return (op.m.size() == 2 && op.m[0] == cplx(1.0) && op.m[1] == cplx(1.0)) ? 1.0 : 6.0;
    default: return 1.0;
  }
}

std::vector<LOp> fuse_greedy(int n, const sv_gate* gates, size_t n_gates, const double* pv, int kmax,
                             std::vector<int>* block_starts, bool dense_always) {
  (void)n;
  std::vector<LOp> out;
  size_t i = 0;
  while (i < n_gates) {
    size_t start = i;
    uint64_t mask = gate_qubit_mask(gates[i]);
    i++;
    if (popc(mask) <= kmax) {
      while (i < n_gates && popc(mask | gate_qubit_mask(gates[i])) <= kmax) {
        mask |= gate_qubit_mask(gates[i]);
        i++;
      }
    }
    if (block_starts) block_starts->push_back((int)start);
    if (i - start == 1) {
      out.push_back(lower_gate(gates[start], pv, (int)start));
      continue;
    }
    // The block's gates, kept (same pass, same result up to rounding) when
    // they cost less than the block's dense matrix.  Below the cost of a real
    // dense block the matrix is not even built: only a block that happened to
    // be diagonal or a permutation could be cheaper.
    std::vector<LOp> parts;
    double parts_cost = 0.0;
    if (!dense_always) {
      for (size_t g = start; g < i; g++) {
        parts.push_back(lower_gate(gates[g], pv, (int)start));
        parts_cost += op_cost(parts.back());
      }
      const int kb = popc(mask);
      if (parts_cost < 4.0 * (1 << kb) + (kb >= 3 ? 40.0 : 2.0)) {
        for (auto& pp : parts) out.push_back(std::move(pp));
        continue;
      }
    }
    // dense block over the union of its gates' qubits, ascending
    LOp op;
    int local_of[64];
    int nb = 0;
    for (int q = 0; q < 64; q++)
      if ((mask >> q) & 1ull) {
        local_of[q] = nb;
        op.q[nb++] = q;
      }
    op.k = nb;
    int d = 1 << nb;
    op.m.assign((size_t)d * d, 0.0);
    std::vector<std::vector<cplx>> mats;
    for (size_t g = start; g < i; g++) mats.push_back(gate_matrix(gates[g], pv));
    std::vector<std::vector<cplx>> cols((size_t)d, std::vector<cplx>((size_t)d, cplx(0.0)));
    for (int c = 0; c < d; c++) cols[c][c] = 1.0;
    for (size_t g = start; g < i; g++)  // gate by gate over every column (same order per column)
      for (int c = 0; c < d; c++) apply_local(cols[c], nb, gates[g], mats[g - start], local_of);
    for (int c = 0; c < d; c++)
      for (int r = 0; r < d; r++) op.m[(size_t)r * d + c] = cols[c][r];
    op.first_gate = (int)start;
    classify(op);
    if (!dense_always) {
      if (parts_cost < op_cost(op)) {
        for (auto& pp : parts) out.push_back(std::move(pp));
        continue;
      }
    }
    out.push_back(std::move(op));
  }
  if (block_starts) block_starts->push_back((int)n_gates);
  return out;
}

static int coef_count(const LOp& op) {
  switch (op.kind) {
    case OPK_DENSE:
    case OPK_REAL: return 1 << (2 * op.k);
    case OPK_DIAG: return 1 << op.k;
    case OPK_ANTIDIAG: return 2;
    default: return 0;
  }
}

std::vector<Sweep> schedule_sweeps(int n, const std::vector<LOp>& ops, int tile_q, int low_q, int coef_pool,
                                   int ops_per_pass) {
  const int max_ops = ops_per_pass > 0 ? std::min(ops_per_pass, kMaxOps) : kMaxOps;
  std::vector<Sweep> out;
  const int m_max = std::min(n, tile_q);
  const int L0 = std::min(n, low_q);
  const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1ull);
  std::vector<char> done(ops.size(), 0);
  size_t first = 0, ndone = 0;
  while (ndone < ops.size()) {
    Sweep sw;
    uint64_t S = (1ull << L0) - 1ull;
    uint64_t blocked = 0;
    int coef = 0;
    for (size_t i = first; i < ops.size(); i++) {
      if (done[i]) continue;
      const LOp& op = ops[i];
      if (op.touch & blocked) {
        blocked |= op.touch;
        if ((blocked & all) == all) break;
        continue;
      }
      uint64_t S2 = S | op.need;
      int c = coef_count(op);
      if (popc(S2) <= m_max && (int)sw.ops.size() < max_ops && coef + c <= coef_pool) {
        S = S2;
        coef += c;
        sw.ops.push_back((int)i);
        done[i] = 1;
        ndone++;
      } else {
        blocked |= op.touch;
        if ((blocked & all) == all) break;
      }
    }
    if (sw.ops.empty()) fail(SV_ERR_INVALID, "scheduler could not place an operation");
    // fill the tile with the lowest remaining qubits (longer contiguous runs)
    for (int q = 0; q < n && popc(S) < m_max; q++) S |= 1ull << q;
    sw.m = 0;
    for (int q = 0; q < n; q++)
      if ((S >> q) & 1ull) sw.tq[sw.m++] = q;
    sw.L = 0;
    while (sw.L < sw.m && sw.tq[sw.L] == sw.L) sw.L++;
    out.push_back(std::move(sw));
    while (first < ops.size() && done[first]) first++;
  }
  return out;
}

// An uncontrolled complex one-qubit op g diag(1, ephi) R diag(1, elam)
// (R = [[C, -S], [S, C]]) becomes two ops: R diag(1, elam), which the program
// builder runs as in-place shears after a phase table, and the closing
// diagonal g diag(1, ephi).  That diagonal is free to move (it commutes with
// everything that does not target the qubit), so it can join the opening
// table of the next gate on the same qubit, possibly in a later pass, instead
// of costing a phase table of its own.  Ops the factors do not reproduce
// within tol stay whole.
static void split_one_qubit(std::vector<LOp>& ops, double tol) {
  // Worth it only where the closing diagonal has a table to join: the next
  // op that targets the qubit (diagonals aside) is another uncontrolled
  // one-qubit gate.  Before a CNOT target, say, it would cost a table anyway.
  auto u1 = [&](const LOp& op) { return (op.kind == OPK_DENSE || op.kind == OPK_REAL) && op.k == 1 && op.nc == 0; };
  std::vector<char> split(ops.size(), 0);
  std::vector<int> next(64, -1);  // per qubit: the next non-diagonal op targeting it
  for (int i = (int)ops.size() - 1; i >= 0; i--) {
    const LOp& op = ops[i];
    if (op.kind == OPK_DIAG) continue;
    if (op.kind == OPK_DENSE && u1(op) && next[op.q[0]] >= 0 && u1(ops[next[op.q[0]]])) split[i] = 1;
    for (int j = 0; j < op.k; j++) next[op.q[j]] = i;
  }
  std::vector<LOp> out;
  out.reserve(ops.size() * 2);
  for (size_t i = 0; i < ops.size(); i++) {
    LOp& op = ops[i];
    RotSplit r;
    if (!(split[i] && rot_split(op.m.data(), tol, r))) {
      out.push_back(std::move(op));
      continue;
    }
    auto part = [&](cplx m00, cplx m01, cplx m10, cplx m11) {
      LOp d;
      d.k = 1;
      d.q[0] = op.q[0];
      d.first_gate = op.first_gate;
      d.m = {m00, m01, m10, m11};
      classify(d);
      return d;
    };
    out.push_back(part(r.C, -r.S * r.elam, r.S, r.C * r.elam));
    out.push_back(part(r.g, 0.0, 0.0, r.g * r.ephi));
  }
  ops = std::move(out);
}

// A narrow diagonal commutes with every op that does not target one of its
// qubits.  One that meets no such op (a "blocker") in the rest of its pass
// moves to the front of the first later pass that holds one -- every pass in
// between leaves its qubits alone -- where the program builder folds it into
// the phase table of its blocker's register phase.  Without a later blocker,
// or without room in that pass, it stays.
static void defer_diagonals(const std::vector<LOp>& ops, std::vector<Sweep>& sw, int max_ops, int coef_pool) {
  auto is_diag = [&](int i) { return ops[i].kind == OPK_DIAG && ops[i].k <= 2; };
  auto targets = [&](int i) {
    uint64_t t = 0;
    for (int j = 0; j < ops[i].k; j++) t |= 1ull << ops[i].q[j];
    return t;
  };
  const size_t ns = sw.size();
  std::vector<int> n_ops(ns), n_coef(ns, 0);
  std::vector<uint64_t> blockers(ns, 0);  // qubits targeted by each pass's non-diagonal ops
  for (size_t s = 0; s < ns; s++) {
    n_ops[s] = (int)sw[s].ops.size();
    for (int i : sw[s].ops) {
      n_coef[s] += coef_count(ops[i]);
      if (!is_diag(i)) blockers[s] |= targets(i);
    }
  }
  std::vector<std::vector<int>> front(ns);  // diagonals arriving at each pass, in order
  for (size_t s = 0; s + 1 < ns; s++) {
    std::vector<int> keep;
    const std::vector<int>& cur = sw[s].ops;
    for (size_t a = 0; a < cur.size(); a++) {
      const int i = cur[a];
      size_t dest = 0;
      if (is_diag(i)) {
        bool blocked_here = false;
        for (size_t b = a + 1; b < cur.size() && !blocked_here; b++)
          blocked_here = !is_diag(cur[b]) && (targets(cur[b]) & ops[i].touch);
        if (!blocked_here)
          for (size_t t = s + 1; t < ns && !dest; t++)
            if (blockers[t] & ops[i].touch) dest = t;
        const int c = coef_count(ops[i]);
        if (dest && (n_ops[dest] + 1 > max_ops || n_coef[dest] + c > coef_pool)) dest = 0;
        if (dest) {
          front[dest].push_back(i);
          n_ops[dest]++;
          n_coef[dest] += c;
          n_ops[s]--;
          n_coef[s] -= c;
        }
      }
      if (!dest) keep.push_back(i);
    }
    sw[s].ops = std::move(keep);
    if (!front[s + 1].empty()) {
      front[s + 1].insert(front[s + 1].end(), sw[s + 1].ops.begin(), sw[s + 1].ops.end());
      sw[s + 1].ops = std::move(front[s + 1]);
    }
  }
}

Plan make_plan(int n, sv_dtype dtype, const sv_gate* gates, size_t n_gates, const double* param_values,
               size_t n_param_values, const sv_exec_opts& opts, int tile_q_override) {
  const int fuse_max_k = opts.fuse_max_k;
  if (opts.block_mode != SV_BLOCK_AUTO && opts.block_mode != SV_BLOCK_DENSE) fail(SV_ERR_INVALID, "unknown block_mode");
  if (opts.ops_per_pass < 0) fail(SV_ERR_INVALID, "ops_per_pass must be >= 0");
  if (opts.tile_qubits != 0 && (opts.tile_qubits < 8 || opts.tile_qubits > (dtype == SV_C64 ? 13 : 11)))
    fail(SV_ERR_INVALID, "tile_qubits must be 0, or 8..13 (complex64) / 8..11 (complex128)");
  if (n < 1 || n > SV_MAX_QUBITS) fail(SV_ERR_INVALID, "n_qubits out of range");
  if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_INVALID, "unknown dtype");
  if (fuse_max_k != 0 && (fuse_max_k < 2 || fuse_max_k > 5))
    fail(SV_ERR_INVALID, "fuse_max_k must be 0 or 2..5 (Sec. 4.3: a positive setting is at least 2)");
  if (n_param_values && !param_values) fail(SV_ERR_INVALID, "param_values is NULL");
  validate_gates(n, gates, n_gates, n_param_values);
  Plan p;
  p.n = n;
  if (fuse_max_k >= 2) {
    p.ops = fuse_greedy(n, gates, n_gates, param_values, fuse_max_k, &p.block_starts,
                        opts.block_mode == SV_BLOCK_DENSE);
  } else {
    p.ops.reserve(n_gates);
    for (size_t i = 0; i < n_gates; i++) {
      p.ops.push_back(lower_gate(gates[i], param_values, (int)i));
      p.block_starts.push_back((int)i);
    }
    p.block_starts.push_back((int)n_gates);
  }
  // drop exact identities (e.g. the I gate): they move no amplitude
  auto drop_identities = [](std::vector<LOp>& ops) {
    std::vector<LOp> kept;
    kept.reserve(ops.size());
    for (auto& op : ops) {
      if (op.kind == OPK_DIAG) {
        bool ident = true;
        for (auto& v : op.m)
          if (v != 1.0) ident = false;
        if (ident) continue;
      }
      kept.push_back(std::move(op));
    }
    ops = std::move(kept);
  };
  drop_identities(p.ops);
  int pool = dtype == SV_C64 ? SweepProgram<float>::kPool : SweepProgram<double>::kPool;
  const int tile_q = tile_q_override > 0 ? tile_q_override
                     : opts.tile_qubits > 0 ? std::min(opts.tile_qubits, n)
                                            : tile_qubits_for(dtype, n);
  const int max_ops = opts.ops_per_pass > 0 ? std::min(opts.ops_per_pass, kMaxOps) : kMaxOps;
  p.sweeps = schedule_sweeps(n, p.ops, tile_q, low_qubits_for(dtype), pool, opts.ops_per_pass);
  if (opts.ops_per_pass != 1) {
    defer_diagonals(p.ops, p.sweeps, max_ops, pool);
    // The split form has more ops, which can cut the greedy passes short and
    // leave more of them: keep it only when it needs no more passes.
    std::vector<LOp> ops2 = p.ops;
    split_one_qubit(ops2, dtype == SV_C64 ? 1e-9 : 1e-13);
    drop_identities(ops2);
    std::vector<Sweep> sw2 = schedule_sweeps(n, ops2, tile_q, low_qubits_for(dtype), pool, opts.ops_per_pass);
    if (sw2.size() <= p.sweeps.size()) {
      defer_diagonals(ops2, sw2, max_ops, pool);
      p.ops = std::move(ops2);
      p.sweeps = std::move(sw2);
    }
  }
  return p;
}

}  // namespace sv
