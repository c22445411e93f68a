// sv_program.cpp -- the pass kernel's programs: turns one sweep of a plan
// (tile qubits and lowered ops, sv_plan.cpp) into the SweepProgram the kernel
// interprets (phases, register slots, rotations, phase tables, dispatch
// words), and runs such programs on the host for validation.
#include <algorithm>
#include <complex>
#include <memory>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <tuple>
#include <vector>

#include "sv_internal.h"

namespace sv {

namespace {

// ----------------------------------------------------------- programs

#ifndef SV_ROT_SPLIT
#define SV_ROT_SPLIT 1
#endif
constexpr bool g_rot_split = SV_ROT_SPLIT != 0;  // register phases in rotation + phase-table form

}  // namespace

// A 2x2 unitary U written as g * diag(1, ephi) * [[C, -S], [S, C]] * diag(1, elam)
// with C = |U00| and S = |U10| (C^2 + S^2 = 1, |g| = |ephi| = |elam| = 1): the
// Z-Y-Z Euler form of a one-qubit gate, C = cos(alpha), S = sin(alpha), alpha
// in [0, pi/2].
bool rot_split(const cplx* U, double tol, RotSplit& r) {
  double C = std::abs(U[0]), S = std::abs(U[2]);
  const double nrm = std::hypot(C, S);
  if (!(nrm > 0.5 && nrm < 2.0)) return false;
  C /= nrm;
  S /= nrm;
  constexpr double tiny = 1e-150;
  const cplx g = std::abs(U[0]) > tiny ? U[0] / std::abs(U[0])
                 : std::abs(U[1]) > tiny ? -U[1] / std::abs(U[1])
                                          : cplx(1.0);
  cplx ephi = 1.0, elam = 1.0;
  if (std::abs(U[2]) > tiny && std::abs(U[1]) > tiny) {
    ephi = (U[2] / std::abs(U[2])) / g;
    elam = -(U[1] / std::abs(U[1])) / g;
  } else if (std::abs(U[3]) > tiny) {  // diagonal
    ephi = (U[3] / std::abs(U[3])) / g;
  }
  // reconstruct and compare
  const cplx M[4] = {g * C, -g * S * elam, g * ephi * S, g * ephi * elam * C};
  for (int i = 0; i < 4; i++)
    if (!(std::abs(M[i] - U[i]) <= tol)) return false;
  r.g = g;
  r.ephi = ephi;
  r.elam = elam;
  r.C = C;
  r.S = S;
  return true;
}

// Converts one sweep of the plan into the kernel's program: each op gets local
// positions and control masks; consecutive ops whose moving qubits fit four
// register slots form one register phase; dense k >= 3 blocks and wide
// diagonals get a shared-memory phase of their own.
template <typename R>
void build_program(const Plan& plan, const Sweep& sw, SweepProgram<R>& P, int rq_override) {
  std::memset(&P.h, 0, sizeof(P.h));
  P.h.n = plan.n;
  P.h.m = sw.m;
  P.h.L = sw.L;
  const int rq = rq_override > 0 ? rq_override : reg_qubits_for(sw.m);
  P.h.rq = rq;
  P.h.nops = (int)sw.ops.size();
  int loc[64];
  for (int q = 0; q < 64; q++) loc[q] = -1;
  for (int i = 0; i < sw.m; i++) {
    P.h.tq[i] = (int8_t)sw.tq[i];
    loc[sw.tq[i]] = i;
  }
  const bool reg_ok = sw.m >= rq && sw.m - rq <= 8;
  struct Tmp {
    DevOp d;
    std::vector<cplx> m;
    bool smem;
    uint32_t need;  // local positions that must be register slots
  };
  // Op order inside the pass.  Diagonal ops commute with each other and with
  // every op whose targets (not controls) avoid their qubits.  A narrow
  // diagonal D may sit anywhere between the last earlier op that targets one
  // of its qubits (a "blocker") and the first later one: every op in between
  // commutes with it, whichever side of D it was on.  It is placed just
  // before its first later blocker, so it lands in the phase where its qubits
  // are register slots and joins that phase's table (attach = +1); the
  // rotation grouping below may hoist it further, in front of a whole group.
  // Without a later blocker it goes just after the run of uncontrolled
  // one-qubit gates that holds its last earlier blocker (attach = -1).
  const int nsw = (int)sw.ops.size();
  std::vector<int> order(nsw), attach(nsw, 0);
  {
    auto is_diag = [&](int i) {
      const LOp& op = plan.ops[sw.ops[i]];
      return op.kind == OPK_DIAG && op.k <= 2;
    };
    auto is_u1 = [&](int i) {
      const LOp& op = plan.ops[sw.ops[i]];
      return (op.kind == OPK_DENSE || op.kind == OPK_REAL) && op.k == 1 && op.nc == 0;
    };
    auto targets = [&](int i) {
      const LOp& op = plan.ops[sw.ops[i]];
      uint64_t t = 0;
      for (int j = 0; j < op.k; j++) t |= 1ull << op.q[j];
      return t;
    };
    // end of the run of uncontrolled one-qubit gates (diagonals skipped) holding each op
    std::vector<int> run_end(nsw);
    int next = -1;
    for (int i = nsw - 1; i >= 0; i--) {
      if (is_diag(i)) continue;
      run_end[i] = (next >= 0 && is_u1(i) && is_u1(next)) ? run_end[next] : i;
      next = i;
    }
    std::vector<std::tuple<int, int, int>> key(nsw);  // (anchor, before/at/after, original index)
    for (int i = 0; i < nsw; i++) {
      key[i] = std::make_tuple(i, 1, i);
      if (!is_diag(i)) continue;
      const uint64_t qs = plan.ops[sw.ops[i]].touch;
      int after = -1, before = -1;
      for (int j = i - 1; j >= 0 && before < 0; j--)
        if (!is_diag(j) && (targets(j) & qs)) before = j;
      for (int j = i + 1; j < nsw && after < 0; j++)
        if (!is_diag(j) && (targets(j) & qs)) after = j;
      if (after >= 0) {
        key[i] = std::make_tuple(after, 0, i);
        attach[i] = 1;
      } else if (before >= 0) {
        key[i] = std::make_tuple(run_end[before], 2, i);
        attach[i] = -1;
      }
    }
    for (int i = 0; i < nsw; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
    if (std::getenv("SV_DEBUG_PLAN") && std::getenv("SV_DEBUG_PLAN")[0] == '3') {
      std::fprintf(stderr, "[sv order]");
      for (int i = 0; i < nsw; i++) {
        const LOp& op = plan.ops[sw.ops[order[i]]];
        std::fprintf(stderr, " %s%d%s%d", is_diag(order[i]) ? "D" : "U", op.q[0], op.k > 1 ? "." : "", op.k > 1 ? op.q[1] : (op.nc ? op.c[0] : -1));
        std::fprintf(stderr, "@%d", order[i]);
      }
      std::fprintf(stderr, "\n");
    }
  }
  std::vector<Tmp> ts(sw.ops.size());
  std::vector<int> ts_attach(nsw);
  for (size_t oi = 0; oi < sw.ops.size(); oi++) {
    const LOp& op = plan.ops[sw.ops[order[oi]]];
    ts_attach[oi] = attach[order[oi]];
    Tmp& t = ts[oi];
    DevOp& d = t.d;
    std::memset(&d, 0, sizeof(d));
    d.kind = op.kind;
    d.k = (uint8_t)op.k;
    t.m = op.m;
    t.need = 0;
    for (int i = 0; i < 5; i++) d.rs[i] = 0xFF;
    int sp[5], ns = 0;
    const bool diag = op.kind == OPK_DIAG;
    for (int i = 0; i < op.k; i++) {
      int l = loc[op.q[i]];
      d.gq[i] = (uint8_t)op.q[i];
      if (diag) {
        d.pos[i] = l < 0 ? 0xFF : (uint8_t)l;
      } else {
        if (l < 0) fail(SV_ERR_INVALID, "internal: target outside the tile");
        d.pos[i] = (uint8_t)l;
        sp[ns++] = l;
        t.need |= 1u << l;
      }
    }
    for (int i = 1; i < ns; i++)
      for (int j = i; j > 0 && sp[j - 1] > sp[j]; j--) std::swap(sp[j], sp[j - 1]);
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
    if (diag) {
      // diag(1, .., 1, -1): a sign flip where every matrix bit is 1 (Z, CZ, CCZ)
      const int dd = 1 << op.k;
      bool sign = true;
      for (int r = 0; r < dd; r++)
        if (op.m[r] != (r == dd - 1 ? cplx(-1.0) : cplx(1.0))) sign = false;
      if (sign) {
        d.kind = OPK_SIGN;
        t.m.clear();
        for (int i = 0; i < op.k; i++) {
          if (d.pos[i] != 0xFF) {
            d.lmask |= 1u << d.pos[i];
            d.lval |= 1u << d.pos[i];
          } else {
            d.xmask |= 1ull << op.q[i];
            d.xval |= 1ull << op.q[i];
          }
        }
      }
    }
    if (op.kind == OPK_ANTIDIAG && op.m.size() == 2 && op.m[0] == cplx(1.0) && op.m[1] == cplx(1.0)) d.pad = 1;
    const bool wide = (op.kind == OPK_DENSE || op.kind == OPK_REAL) ? op.k >= 3 : (diag && d.kind == OPK_DIAG && op.k >= 3);
    t.smem = !reg_ok || wide;
  }

  // phases
  int nph = 0;
  auto add_phase = [&](PhaseKind kind, int first, int nops, uint32_t need) {
    if (nph >= kMaxPhases) fail(SV_ERR_INVALID, "internal: too many phases");
    Phase& ph = P.ph[nph++];
    std::memset(&ph, 0, sizeof(ph));
    ph.kind = kind;
    ph.first = (uint8_t)first;
    ph.nops = (uint8_t)nops;
    if (kind != PH_REG) return;
    // register slots: the needed positions, then local bit 0 (16-byte
    // shared-memory accesses), then the highest free positions
    uint32_t rp = need;
    if (__builtin_popcount(rp) < rq && !(rp & 1u)) rp |= 1u;
    for (int q = sw.m - 1; q >= 0 && __builtin_popcount(rp) < rq; q--) rp |= 1u << q;
    int slot_of[32];
    int ns2 = 0, nt = 0;
    for (int q = 0; q < sw.m; q++) {
      if ((rp >> q) & 1u) {
        slot_of[q] = ns2;
        ph.rp[ns2++] = (uint8_t)q;
      } else {
        slot_of[q] = -1;
        ph.tpos[nt++] = (uint8_t)q;
      }
    }
    ph.ntpos = (uint8_t)nt;
    ph.nrp = (uint8_t)ns2;
    for (int o = first; o < first + nops; o++) {
      Tmp& t = ts[o];
      DevOp& d = t.d;
      for (int i = 0; i < d.k; i++)
        d.rs[i] = (d.pos[i] != 0xFF && slot_of[d.pos[i]] >= 0) ? (uint8_t)slot_of[d.pos[i]] : 0xFF;
      d.rmask = d.rval = 0;
      d.tmask = d.tval = 0;
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
      // two-qubit register ops want rs[0] < rs[1]: swap the matrix qubit order
      if (d.k == 2 && d.kind != OPK_DIAG && d.kind != OPK_SIGN && d.rs[0] > d.rs[1]) {
        std::swap(d.rs[0], d.rs[1]);
        std::swap(d.pos[0], d.pos[1]);
        std::swap(d.gq[0], d.gq[1]);
        if (t.m.size() == 16) {
          std::vector<cplx> mt(16);
          auto sw2 = [](int x) { return ((x & 1) << 1) | ((x >> 1) & 1); };
          for (int r = 0; r < 4; r++)
            for (int c = 0; c < 4; c++) mt[r * 4 + c] = t.m[sw2(r) * 4 + sw2(c)];
          t.m = mt;
        }
      }
    }
  };
  // Greedy register phases.  Diagonals attached forward wait for their op and
  // open its phase with it; the others join the phase in progress.
  int cur_first = -1, cur_n = 0, pend = 0;
  uint32_t cur_need = 0;
  for (int o = 0; o < (int)ts.size(); o++) {
    if (ts[o].smem) {
      cur_n += pend;
      pend = 0;
      if (cur_n) add_phase(PH_REG, cur_first, cur_n, cur_need);
      cur_n = 0;
      cur_need = 0;
      add_phase(PH_SMEM, o, 1, 0);
      continue;
    }
    if (ts_attach[o] > 0 && !ts[o].need) {  // waits for the op it was moved in front of
      if (!cur_n && !pend) cur_first = o;
      pend++;
      continue;
    }
    if ((cur_n || pend) && __builtin_popcount(cur_need | ts[o].need) <= rq && cur_n + pend < 255) {
      cur_need |= ts[o].need;
      cur_n += pend + 1;
    } else {
      if (cur_n) add_phase(PH_REG, cur_first, cur_n, cur_need);
      cur_first = o - pend;
      cur_n = pend + 1;
      cur_need = ts[o].need;
    }
    pend = 0;
  }
  cur_n += pend;
  if (cur_n) add_phase(PH_REG, cur_first, cur_n, cur_need);
  P.h.nphases = nph;

  // Final op list.  In a register phase, a run of uncontrolled one-qubit
  // gates is merged per slot (same-slot matrices multiplied in double; distinct
  // slots commute).  Each merged 2x2 unitary is split as
  //   g * diag(1, e^{i phi}) * [[C, -S], [S, C]] * diag(1, e^{i lambda})
  // and the rotations of the run become one KROT op (three in-place shears
  // per slot).  The diagonal factors, the global phases, and every diagonal
  // op on register slots only (Z/CZ sign flips,
  // phase gates) are collected in a table of 2^rq phases over the register
  // combinations.  The table is applied (OPK_PHASE) only when a
  // non-diagonal op needs it: when the table varies along one of the op's
  // target slots (a diagonal commutes with an op whose targets it does not
  // depend on, controls included), and at the end of the phase.  A unitary
  // that does not split within the precision's tolerance falls back to the
  // dense KRON form.  Sign flips involving thread or outside-tile bits carry
  // their pattern of register combinations; flags tell the kernel which
  // control tests to make.
  auto u1_free = [](const Tmp& t) {
    return (t.d.kind == OPK_DENSE || t.d.kind == OPK_REAL) && t.d.k == 1 && t.d.lmask == 0 && t.d.xmask == 0;
  };
  auto pattern = [rq](uint32_t rmask, uint32_t rval) {
    uint32_t p = 0;
    for (int j = 0; j < (1 << rq); j++)
      if (((uint32_t)j & rmask) == rval) p |= 1u << j;
    return p;
  };
  const double split_tol = sizeof(R) == 4 ? 1e-9 : 1e-13;
  std::vector<std::pair<int, int>> span(nph);
  for (int p = 0; p < nph; p++) span[p] = {P.ph[p].first, P.ph[p].nops};
  std::vector<Tmp> fin;
  fin.reserve(2 * ts.size() + 2 * nph);
  auto blank = [](OpKind kind) {
    Tmp t;
    std::memset(&t.d, 0, sizeof(t.d));
    t.d.kind = kind;
    for (int i = 0; i < 5; i++) t.d.rs[i] = 0xFF;
    t.smem = false;
    t.need = 0;
    return t;
  };
  // Per-slot products of uncontrolled one-qubit gates, in order.
  auto merge_ops = [&](const std::vector<int>& list, std::vector<cplx>& mats) {
    mats.assign(4 * rq, 0.0);
    for (int s2 = 0; s2 < rq; s2++) mats[4 * s2] = mats[4 * s2 + 3] = 1.0;
    uint32_t present = 0;
    for (int o : list) {
      const int sl = ts[o].d.rs[0];
      const std::vector<cplx>& U = ts[o].m;
      cplx* M = &mats[4 * sl];
      const cplx a = U[0] * M[0] + U[1] * M[2], b = U[0] * M[1] + U[1] * M[3];
      const cplx c = U[2] * M[0] + U[3] * M[2], d = U[2] * M[1] + U[3] * M[3];
      M[0] = a; M[1] = b; M[2] = c; M[3] = d;
      present |= 1u << sl;
    }
    return present;
  };
  auto kron_op = [&](uint32_t present, const std::vector<cplx>& mats) {
    Tmp k = blank(OPK_KRON);
    k.d.rmask = (uint8_t)present;
    k.m = mats;
    return k;
  };
  auto emit_phase_plain = [&](int first, int nops) {
    for (int o = first; o < first + nops;) {
      if (u1_free(ts[o]) && o + 1 < first + nops && u1_free(ts[o + 1])) {
        int end = o;
        while (end < first + nops && u1_free(ts[end])) end++;
        std::vector<int> list;
        for (int x = o; x < end; x++) list.push_back(x);
        std::vector<cplx> mats;
        const uint32_t present = merge_ops(list, mats);
        fin.push_back(kron_op(present, mats));
        o = end;
      } else {
        fin.push_back(ts[o]);
        o++;
      }
    }
  };
  // max_sel: how many selector bits (thread bits or bits outside the tile) a
  // table may depend on; sign flips and diagonals on such bits fold into the
  // table as 2^nsel variants, picked per thread.
  auto emit_phase_rot = [&](int first, int nops, int max_sel) {
    const int NT = 1 << rq;
    std::vector<int> sel;              // selector codes: local position p, or 64 + global qubit
    std::vector<cplx> tab(NT, 1.0);    // [variant][register combination]
    cplx sc = 1.0;
    auto nvar = [&] { return 1 << (int)sel.size(); };
    auto tab_dep = [&](uint32_t slots) {
      for (int v = 0; v < nvar(); v++)
        for (int j = 0; j < NT; j++)
          for (int s2 = 0; s2 < rq; s2++)
            if (((slots >> s2) & 1u) && tab[v * NT + j] != tab[v * NT + (j ^ (1 << s2))]) return true;
      return false;
    };
    auto flush = [&]() {
      bool id = sc == cplx(1.0);
      for (const cplx& x : tab)
        if (x != cplx(1.0)) id = false;
      if (!id) {
        Tmp t = blank(OPK_PHASE);
        t.d.k = (uint8_t)sel.size();
        for (size_t i = 0; i < sel.size(); i++) t.d.gq[i] = (uint8_t)sel[i];
        const int stride = table_stride<R>(rq);  // padded: variants start in different banks
        t.m.assign((size_t)nvar() * stride, 0.0);
        for (int v = 0; v < nvar(); v++)
          for (int j = 0; j < NT; j++) t.m[v * stride + j] = tab[v * NT + j] * sc;
        fin.push_back(t);
      }
      sel.clear();
      tab.assign(NT, 1.0);
      sc = 1.0;
    };
    // Selector index of `code`, adding it (the table doubles) if there is room.
    auto selector = [&](int code) {
      for (size_t i = 0; i < sel.size(); i++)
        if (sel[i] == code) return (int)i;
      if ((int)sel.size() >= max_sel) return -1;
      const int nv = nvar();
      tab.resize((size_t)2 * nv * NT);
      for (int x = 0; x < nv * NT; x++) tab[nv * NT + x] = tab[x];
      sel.push_back(code);
      return (int)sel.size() - 1;
    };
    // The selectors a diagonal op needs: its thread-bit and outside-tile
    // controls and matrix bits.  Returns false if they cannot all be present.
    auto need_codes = [&](const DevOp& d, std::vector<int>& codes) {
      codes.clear();
      for (int q = 0; q < 32; q++)
        if ((d.tmask >> q) & 1u) codes.push_back(q);
      for (int q = 0; q < 64; q++)
        if ((d.xmask >> q) & 1ull) codes.push_back(64 + q);
      if (d.kind == OPK_DIAG)
        for (int i = 0; i < d.k; i++)
          if (d.rs[i] == 0xFF) codes.push_back(d.pos[i] != 0xFF ? (int)d.pos[i] : 64 + (int)d.gq[i]);
      int fresh = 0;
      for (int c : codes) {
        bool have = false;
        for (int x : sel) have = have || x == c;
        fresh += have ? 0 : 1;
      }
      return (int)sel.size() + fresh <= max_sel;  // otherwise the op stays a sign/diagonal op
    };
    // Folds a sign flip or diagonal into the table (variants included).
    auto fold_diag = [&](const Tmp& t) {
      const DevOp& d = t.d;
      std::vector<int> codes;
      if (!need_codes(d, codes)) return false;
      auto sel_bit = [&](int code, int v) { return (v >> selector(code)) & 1; };
      for (int c : codes) selector(c);  // make sure every needed selector exists
      for (int v = 0; v < nvar(); v++) {
        bool on = true;
        for (int q = 0; q < 32; q++)
          if ((d.tmask >> q) & 1u) on = on && sel_bit(q, v) == (int)((d.tval >> q) & 1u);
        for (int q = 0; q < 64; q++)
          if ((d.xmask >> q) & 1ull) on = on && sel_bit(64 + q, v) == (int)((d.xval >> q) & 1ull);
        if (!on) continue;
        for (int j = 0; j < NT; j++) {
          if (((uint32_t)j & d.rmask) != d.rval) continue;
          cplx& x = tab[v * NT + j];
          if (d.kind == OPK_SIGN) {
            x = -x;
          } else {
            int idx = 0;
            for (int i = 0; i < d.k; i++) {
              int b;
              if (d.rs[i] != 0xFF)
                b = (j >> d.rs[i]) & 1;
              else
                b = sel_bit(d.pos[i] != 0xFF ? (int)d.pos[i] : 64 + (int)d.gq[i], v);
              idx |= b << i;
            }
            x *= t.m[idx];
          }
        }
      }
      return true;
    };
    // A diagonal whose selectors do not fit the current table starts a new
    // one (the current table is emitted first: diagonals commute), so that it
    // stays a table entry instead of a general diagonal op.  Sign flips that
    // do not fit stay sign ops (a negation mask).
    auto fold_or_restart = [&](const Tmp& t) {
      if (fold_diag(t)) return true;
      if (t.d.kind != OPK_DIAG || sel.empty()) return false;
      flush();
      return fold_diag(t);
    };
    for (int o = first; o < first + nops;) {
      const Tmp& t = ts[o];
      const DevOp& d = t.d;
      if (u1_free(t)) {
        // A group of uncontrolled one-qubit gates.  A sign flip or diagonal
        // met on the way that touches no slot rotated so far in the group
        // commutes with the group's earlier gates: it is hoisted in front.
        std::vector<int> list, hoist;
        uint32_t rotated = 0;
        int end = o;
        for (; end < first + nops; end++) {
          const Tmp& u = ts[end];
          if (u1_free(u)) {
            list.push_back(end);
            rotated |= 1u << u.d.rs[0];
            continue;
          }
          if (u.d.kind != OPK_SIGN && u.d.kind != OPK_DIAG) break;
          uint32_t slots = u.d.rmask;
          for (int i = 0; i < u.d.k; i++)
            if (u.d.rs[i] != 0xFF) slots |= 1u << u.d.rs[i];
          if (slots & rotated) break;
          hoist.push_back(end);
        }
        for (int h : hoist)
          if (!fold_or_restart(ts[h])) fin.push_back(ts[h]);
        std::vector<cplx> mats;
        const uint32_t present = merge_ops(list, mats);
        o = end;
        RotSplit sp[kMaxRegQ];
        bool ok = true;
        for (int s2 = 0; s2 < rq; s2++)
          if ((present >> s2) & 1u) ok = ok && rot_split(&mats[4 * s2], split_tol, sp[s2]);
        if (!ok) {
          if (tab_dep(present)) flush();
          fin.push_back(kron_op(present, mats));
          continue;
        }
        for (int s2 = 0; s2 < rq; s2++) {
          if (!((present >> s2) & 1u)) continue;
          for (int x = 0; x < nvar() * NT; x++)
            if ((x >> s2) & 1) tab[x] *= sp[s2].elam;  // bit s2 of x is bit s2 of j (NT = 2^rq)
          sc *= sp[s2].g;
        }
        // complex128 takes the scaled form (two multiply-adds per component),
        // which leaves every amplitude multiplied by max(C, S) per rotated
        // slot, a factor the table carries; complex64 takes three shears (one
        // packed FMA each, no factor).  The scaled form measured slower for
        // complex64 on GB300 (6.00 against 5.65 ms per 30-qubit pass): its
        // per-slot form test and extra temporaries cost more, at the kernel's
        // 128-register budget, than the packed FMA per pair it saves.
        const bool scaled = sizeof(R) == 8;
        if (scaled)
          for (int s2 = 0; s2 < rq; s2++)
            if ((present >> s2) & 1u) sc *= std::max(sp[s2].C, sp[s2].S);
        if (tab_dep(present)) flush();
        Tmp k = blank(OPK_KROT);
        k.d.rmask = (uint8_t)present;
        k.m.assign(rq, 0.0);
        for (int s2 = 0; s2 < rq; s2++) {
          if (!((present >> s2) & 1u)) continue;
          const double C = sp[s2].C, S = sp[s2].S;
          if (!scaled) {         // three shears: (tan(alpha/2), sin(alpha))
            k.m[s2] = cplx(S / (1.0 + C), S);
          } else if (C >= S) {   // scaled form (a - t b, b + t a), t = S/C
            k.m[s2] = S / C;
          } else {               // (t a - b, a + t b), t = C/S
            k.m[s2] = C / S;
            k.d.rval |= (uint8_t)(1u << s2);
          }
        }
        fin.push_back(k);
        for (int s2 = 0; s2 < rq; s2++) {
          if (!((present >> s2) & 1u)) continue;
          for (int x = 0; x < nvar() * NT; x++)
            if ((x >> s2) & 1) tab[x] *= sp[s2].ephi;
        }
        // the scaled form lets the amplitudes grow by up to sqrt(2) per rotation
        if (std::abs(sc) < 1e-30) flush();
        continue;
      }
      if ((d.kind == OPK_SIGN || d.kind == OPK_DIAG) && fold_or_restart(t)) {
        o++;
        continue;
      }
      if (d.kind != OPK_SIGN && d.kind != OPK_DIAG) {
        uint32_t tg = 0;
        for (int i = 0; i < d.k; i++)
          if (d.rs[i] != 0xFF) tg |= 1u << d.rs[i];
        if (tab_dep(tg)) flush();
      }
      fin.push_back(t);
      o++;
    }
    flush();
  };
  // Builds the whole list; false if it does not fit the program (the table
  // form can need more ops and coefficients than the plain one).
  auto make_fin = [&](bool rot, int max_sel) {
    fin.clear();
    size_t ncoef = 0;
    for (int p = 0; p < nph; p++) {
      Phase& ph = P.ph[p];
      const int first = span[p].first, nops = span[p].second;
      const int nf = (int)fin.size();
      if (ph.kind == PH_SMEM) {
        fin.push_back(ts[first]);
      } else {
        if (rot)
          emit_phase_rot(first, nops, max_sel);
        else
          emit_phase_plain(first, nops);
        for (int i = nf; i < (int)fin.size(); i++) {
          DevOp& d = fin[i].d;
          d.pad &= OPF_FLIP;
          if (d.kind != OPK_KRON && d.kind != OPK_KROT && d.kind != OPK_PHASE) {
            if (d.tmask) d.pad |= OPF_TCOND;
            if (d.xmask) d.pad |= OPF_XCOND;
          }
        }
      }
      if ((int)fin.size() - nf > 255) return false;
      ph.first = (uint8_t)nf;
      ph.nops = (uint8_t)((int)fin.size() - nf);
    }
    for (const Tmp& t : fin) ncoef += t.m.size() + (t.d.kind == OPK_PHASE ? 1 : 0);  // + alignment padding
    return (int)fin.size() <= kMaxOps && ncoef <= (size_t)SweepProgram<R>::kPool;
  };
  if (!make_fin(g_rot_split, 3) && !make_fin(g_rot_split, 2) && !make_fin(g_rot_split, 0) && !make_fin(false, 0))
    fail(SV_ERR_INVALID, "internal: program too long");
  P.h.nops = (int)fin.size();

  int coef = 0;
  for (size_t oi = 0; oi < fin.size(); oi++) {
    if (fin[oi].d.kind == OPK_PHASE && sizeof(R) == 4 && (coef & 1)) {  // tables are read in 16-byte pairs
      if (coef >= SweepProgram<R>::kPool) fail(SV_ERR_INVALID, "internal: coefficient pool overflow");
      P.coef[coef].re = P.coef[coef].im = (R)0;
      coef++;
    }
    fin[oi].d.coef = (uint32_t)coef;
    for (const cplx& v : fin[oi].m) {
      if (coef >= SweepProgram<R>::kPool) fail(SV_ERR_INVALID, "internal: coefficient pool overflow");
      P.coef[coef].re = (R)v.real();
      P.coef[coef].im = (R)v.imag();
      coef++;
    }
    P.ops[oi] = fin[oi].d;
  }
  static_assert(SweepProgram<double>::kPool < kCodeCoefMax && SweepProgram<float>::kPool < kCodeCoefMax,
                "coefficient offsets must fit the dispatch word");
  for (int p = 0; p < nph; p++)
    if (P.ph[p].kind == PH_REG)
      for (int o = P.ph[p].first; o < P.ph[p].first + P.ph[p].nops; o++) {
        DevOp& d = P.ops[o];
        if (d.kind == OPK_SIGN) {
          d.coef = pattern(d.rmask, d.rval);
          d.pad = op_code(d.kind, d.pad & 7u, 0, 0, 0);
        } else {
          d.pad = op_code(d.kind, d.pad & 7u, d.rmask, d.rval, d.coef);
        }
      }
  P.h.ncoef = coef;
  static const bool debug = std::getenv("SV_DEBUG_PLAN") != nullptr;
  if (debug) {
    std::fprintf(stderr, "[sv plan] sweep m=%d L=%d tq=", sw.m, sw.L);
    for (int i = 0; i < sw.m; i++) std::fprintf(stderr, "%s%d", i ? "," : "", sw.tq[i]);
    std::fprintf(stderr, " ops=%d phases=%d:", P.h.nops, nph);
    for (int p = 0; p < nph; p++) {
      std::fprintf(stderr, " %s(", P.ph[p].kind == PH_REG ? "R" : "S");
      for (int o = P.ph[p].first; o < P.ph[p].first + P.ph[p].nops; o++)
        std::fprintf(stderr, "%s%d%s", o > P.ph[p].first ? "," : "", (int)P.ops[o].kind, P.ops[o].k > 1 ? "w" : "");
      if (std::getenv("SV_DEBUG_PLAN")[0] == '2') {
        std::fprintf(stderr, " [rp");
        for (int i = 0; i < P.ph[p].nrp; i++) std::fprintf(stderr, " %d", P.h.tq[P.ph[p].rp[i]]);
        std::fprintf(stderr, " | krot masks");
        for (int o = P.ph[p].first; o < P.ph[p].first + P.ph[p].nops; o++)
          if (P.ops[o].kind == OPK_KROT) std::fprintf(stderr, " %x", (P.ops[o].pad >> 7) & 31u);
        std::fprintf(stderr, "]");
      }
      std::fprintf(stderr, ")");
    }
    std::fprintf(stderr, "\n");
  }
}

template void build_program<float>(const Plan&, const Sweep&, SweepProgram<float>&, int);
template void build_program<double>(const Plan&, const Sweep&, SweepProgram<double>&, int);

}  // namespace sv

// ----------------------------------------------------------------- host execution
//
// The programs above run on the host exactly as the pass kernel reads them
// (dispatch words, register slots, table variants, shears or scaled
// rotations, sign patterns, shared-memory ops), in double precision.  This
// checks the program builder against the oracle without a GPU; it says
// nothing about the kernel's own arithmetic.

namespace sv {
namespace {

using zc = std::complex<double>;

inline uint32_t ins0h(uint32_t x, int p) { return ((x >> p) << (p + 1)) | (x & ((1u << p) - 1u)); }

template <typename R>
zc cz(const Cx<R>& c) {
  return zc((double)c.re, (double)c.im);
}

template <typename R>
void emulate_reg_op(const SweepProgram<R>& P, const DevOp& op, uint32_t code, int rq, std::vector<zc>& v,
                    uint32_t tb, uint64_t base) {
  const int NR = 1 << rq;
  const uint32_t fl = (code >> 4) & 7u;
  if ((fl & OPF_XCOND) && (base & op.xmask) != op.xval) return;
  if ((fl & OPF_TCOND) && (tb & op.tmask) != op.tval) return;
  const Cx<R>* cf = P.coef + (code >> 17);
  const uint32_t rm = (code >> 7) & 31u, rv = (code >> 12) & 31u;
  auto pairs = [&](int S, bool use_controls, auto&& f) {
    for (int j = 0; j < NR; j++) {
      if (j & (1 << S)) continue;
      if (use_controls && ((uint32_t)j & rm) != rv) continue;
      f(v[j], v[j | (1 << S)]);
    }
  };
  switch (code & 15u) {
    case OPK_KRON:
      for (int S = 0; S < rq; S++)
        if ((rm >> S) & 1u)
          pairs(S, false, [&](zc& a, zc& b) {
            const zc a0 = a, b0 = b;
            a = cz(cf[4 * S]) * a0 + cz(cf[4 * S + 1]) * b0;
            b = cz(cf[4 * S + 2]) * a0 + cz(cf[4 * S + 3]) * b0;
          });
      break;
    case OPK_KROT:
      for (int S = 0; S < rq; S++) {
        if (!((rm >> S) & 1u)) continue;
        const double t = (double)cf[S].re, sn = (double)cf[S].im;
        const bool cot = (rv >> S) & 1u;
        const bool shears = sizeof(R) == 4;
        pairs(S, false, [&](zc& a, zc& b) {
          if (shears) {
            a -= t * b;
            b += sn * a;
            a -= t * b;
          } else if (cot) {
            const zc a0 = a;
            a = t * a0 - b;
            b = a0 + t * b;
          } else {
            const zc a0 = a;
            a = a0 - t * b;
            b = b + t * a0;
          }
        });
      }
      break;
    case OPK_PHASE: {
      uint32_t var = 0;
      for (int i = 0; i < op.k; i++) {
        const uint32_t c = op.gq[i];
        const uint32_t bit = c < 64 ? (tb >> c) & 1u : (uint32_t)(base >> (c - 64)) & 1u;
        var |= bit << i;
      }
      for (int j = 0; j < NR; j++) v[j] *= cz(cf[var * table_stride<R>(rq) + j]);
      break;
    }
    case OPK_DENSE:
    case OPK_REAL:
      if (op.k == 1) {
        pairs(op.rs[0], true, [&](zc& a, zc& b) {
          const zc a0 = a, b0 = b;
          a = cz(cf[0]) * a0 + cz(cf[1]) * b0;
          b = cz(cf[2]) * a0 + cz(cf[3]) * b0;
        });
      } else {
        const int A = op.rs[0], B = op.rs[1];
        for (int j = 0; j < NR; j++) {
          if (j & ((1 << A) | (1 << B))) continue;
          if (((uint32_t)j & rm) != rv) continue;
          const int idx[4] = {j, j | (1 << A), j | (1 << B), j | (1 << A) | (1 << B)};
          zc x[4], y[4];
          for (int c = 0; c < 4; c++) x[c] = v[idx[c]];
          for (int r = 0; r < 4; r++) {
            y[r] = 0.0;
            for (int c = 0; c < 4; c++) y[r] += cz(cf[r * 4 + c]) * x[c];
          }
          for (int r = 0; r < 4; r++) v[idx[r]] = y[r];
        }
      }
      break;
    case OPK_ANTIDIAG:
      pairs(op.rs[0], true, [&](zc& a, zc& b) {
        const zc a0 = a, b0 = b;
        if (fl & OPF_FLIP) {
          a = b0;
          b = a0;
        } else {
          a = cz(cf[0]) * b0;
          b = cz(cf[1]) * a0;
        }
      });
      break;
    case OPK_SWAP: {
      const int A = op.rs[0], B = op.rs[1];
      for (int j = 0; j < NR; j++) {
        if (j & ((1 << A) | (1 << B))) continue;
        if (((uint32_t)j & rm) != rv) continue;
        std::swap(v[j | (1 << A)], v[j | (1 << B)]);
      }
      break;
    }
    case OPK_DIAG: {
      uint32_t dbase = 0;
      for (int i = 0; i < op.k; i++) {
        if (op.rs[i] != 0xFF) continue;
        const uint32_t bit = op.pos[i] != 0xFF ? (tb >> op.pos[i]) & 1u : (uint32_t)(base >> op.gq[i]) & 1u;
        dbase |= bit << i;
      }
      for (int j = 0; j < NR; j++) {
        if (((uint32_t)j & op.rmask) != op.rval) continue;
        uint32_t idx = dbase;
        for (int i = 0; i < op.k; i++)
          if (op.rs[i] != 0xFF) idx |= (uint32_t)((j >> op.rs[i]) & 1) << i;
        v[j] *= cz(cf[idx]);
      }
      break;
    }
    default:
      fail(SV_ERR_INVALID, "internal: unknown register op");
  }
}

template <typename R>
void emulate_smem_op(const SweepProgram<R>& P, const DevOp& op, std::vector<zc>& s, uint64_t base) {
  if ((base & op.xmask) != op.xval) return;
  const int tsz = (int)s.size();
  const Cx<R>* cf = P.coef + op.coef;
  if (op.kind == OPK_DIAG || op.kind == OPK_SIGN) {
    uint32_t xi = 0;
    for (int i = 0; i < op.k; i++)
      if (op.pos[i] == 0xFF) xi |= (uint32_t)((base >> op.gq[i]) & 1ull) << i;
    for (int a = 0; a < tsz; a++) {
      if (((uint32_t)a & op.lmask) != op.lval) continue;
      if (op.kind == OPK_SIGN) {
        s[a] = -s[a];
      } else {
        uint32_t di = xi;
        for (int i = 0; i < op.k; i++)
          if (op.pos[i] != 0xFF) di |= (((uint32_t)a >> op.pos[i]) & 1u) << i;
        s[a] *= cz(cf[di]);
      }
    }
  } else if (op.kind == OPK_ANTIDIAG) {
    const int p = op.pos[0];
    for (int g = 0; g < tsz / 2; g++) {
      const uint32_t i0 = ins0h((uint32_t)g, p), i1 = i0 | (1u << p);
      if ((i0 & op.lmask) != op.lval) continue;
      const zc x = s[i0], y = s[i1];
      s[i0] = cz(cf[0]) * y;
      s[i1] = cz(cf[1]) * x;
    }
  } else if (op.kind == OPK_SWAP) {
    for (int g = 0; g < tsz / 4; g++) {
      const uint32_t b = ins0h(ins0h((uint32_t)g, op.spos[0]), op.spos[1]);
      if ((b & op.lmask) != op.lval) continue;
      std::swap(s[b | (1u << op.pos[0])], s[b | (1u << op.pos[1])]);
    }
  } else {  // dense k
    const int K = op.k, D = 1 << K;
    std::vector<zc> x(D), y(D);
    for (int g = 0; g < (tsz >> K); g++) {
      uint32_t b = (uint32_t)g;
      for (int i = 0; i < K; i++) b = ins0h(b, op.spos[i]);
      if ((b & op.lmask) != op.lval) continue;
      auto at = [&](int j) {
        uint32_t a = b;
        for (int i = 0; i < K; i++)
          if ((j >> i) & 1) a |= 1u << op.pos[i];
        return a;
      };
      for (int j = 0; j < D; j++) x[j] = s[at(j)];
      for (int r = 0; r < D; r++) {
        y[r] = 0.0;
        for (int c = 0; c < D; c++) y[r] += cz(cf[r * D + c]) * x[c];
      }
      for (int r = 0; r < D; r++) s[at(r)] = y[r];
    }
  }
}

template <typename R>
void emulate_program(const SweepProgram<R>& P, zc* state) {
  const ProgramHeader& h = P.h;
  const int m = h.m, tsz = 1 << m, rq = h.rq;
  std::vector<zc> s(tsz), v(1 << rq);
  for (uint64_t tile = 0; tile < (1ull << (h.n - m)); tile++) {
    uint64_t base = tile;
    for (int i = 0; i < m; i++) base = ((base >> h.tq[i]) << (h.tq[i] + 1)) | (base & ((1ull << h.tq[i]) - 1ull));
    auto global = [&](uint32_t l) {
      uint64_t g = base;
      for (int i = 0; i < m; i++)
        if ((l >> i) & 1u) g |= 1ull << h.tq[i];
      return g;
    };
    for (int l = 0; l < tsz; l++) s[l] = state[global((uint32_t)l)];
    for (int p = 0; p < h.nphases; p++) {
      const Phase& ph = P.ph[p];
      if (ph.kind != PH_REG) {
        emulate_smem_op(P, P.ops[ph.first], s, base);
        continue;
      }
      for (uint32_t t = 0; t < (1u << ph.ntpos); t++) {
        uint32_t tb = t;
        for (int i = 0; i < rq; i++) tb = ins0h(tb, ph.rp[i]);
        auto slot = [&](int j) {
          uint32_t a = tb;
          for (int i = 0; i < rq; i++)
            if ((j >> i) & 1) a |= 1u << ph.rp[i];
          return a;
        };
        for (int j = 0; j < (1 << rq); j++) v[j] = s[slot(j)];
        uint32_t neg = 0;
        for (int o = ph.first; o < ph.first + ph.nops; o++) {
          const DevOp& op = P.ops[o];
          const uint32_t code = op.pad;
          if ((code & 15u) == OPK_SIGN) {
            bool on = true;
            if (code & (OPF_XCOND << 4)) on = (base & op.xmask) == op.xval;
            if (code & (OPF_TCOND << 4)) on = on && (tb & op.tmask) == op.tval;
            if (on) neg ^= op.coef;
            continue;
          }
          for (int j = 0; j < (1 << rq); j++)
            if ((neg >> j) & 1u) v[j] = -v[j];
          neg = 0;
          emulate_reg_op(P, op, code, rq, v, tb, base);
        }
        for (int j = 0; j < (1 << rq); j++)
          if ((neg >> j) & 1u) v[j] = -v[j];
        for (int j = 0; j < (1 << rq); j++) s[slot(j)] = v[j];
      }
    }
    for (int l = 0; l < tsz; l++) state[global((uint32_t)l)] = s[l];
  }
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_emulate_apply(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                                      const double* param_values, size_t n_param_values, const sv_exec_opts* opts,
                                      double* state) {
  return guarded([&] {
    if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_INVALID, "unknown dtype");
    if (n_qubits < 1 || n_qubits > 20) fail(SV_ERR_INVALID, "host execution takes 1..20 qubits");
    if (!state) fail(SV_ERR_INVALID, "state is NULL");
    if (n_gates && !gates) fail(SV_ERR_INVALID, "gates is NULL");
    sv_exec_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    const Plan plan = make_plan(n_qubits, dtype, gates, n_gates, param_values, n_param_values, o);
    zc* st = reinterpret_cast<zc*>(state);
    if (dtype == SV_C64) {
      std::unique_ptr<SweepProgram<float>> P(new SweepProgram<float>());
      for (const Sweep& sw : plan.sweeps) {
        build_program<float>(plan, sw, *P);
        emulate_program<float>(*P, st);
      }
    } else {
      std::unique_ptr<SweepProgram<double>> P(new SweepProgram<double>());
      for (const Sweep& sw : plan.sweeps) {
        build_program<double>(plan, sw, *P);
        emulate_program<double>(*P, st);
      }
    }
  });
}
