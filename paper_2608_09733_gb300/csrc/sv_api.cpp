// sv_api.cpp -- the extern "C" boundary declared in include/sv.h.
//
// Every entry point validates its arguments on the host before it touches the
// device (Sec. 3.3: unsupported combinations raise at their boundary; the
// distributed path likewise checks before allocating), converts the gate
// records into device programs and launches the kernels on the caller's
// stream.  Device pointers are checked to be device (or managed) memory of the
// current device, 16-byte aligned and, where the driver reports the owning
// allocation, large enough for 2^n amplitudes, so that a wrong pointer or size
// is an error status rather than an out-of-bounds access.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "sv_internal.h"

namespace sv {
namespace {

thread_local std::string g_last_error;

size_t amp_bytes(sv_dtype d) { return d == SV_C64 ? 8 : 16; }

void check_dtype_n(int n, sv_dtype dtype) {
  if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_INVALID, "unknown dtype");
  if (n < 1 || n > SV_MAX_QUBITS) fail(SV_ERR_INVALID, "n_qubits must be in 1..34");
}

// cuMemGetAddressRange through the runtime's driver entry point (no link-time
// dependency on libcuda).
using AddrRangeFn = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);
AddrRangeFn addr_range_fn() {
  static AddrRangeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (AddrRangeFn) nullptr;
    }
    return (AddrRangeFn)p;
  }();
  return fn;
}

}  // namespace

void set_last_error(const std::string& m) { g_last_error = m; }

// Waits for the stream; a pass kernel that gave up on its tile copies is
// reported here as well.
void sync_stream(cudaStream_t s) {
  cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (sweep_timed_out())
    fail(SV_ERR_TIMEOUT, "a pass gave up waiting (2 s) for its tile copies; the state is not valid");
}

void check_device_buffer(const void* p, size_t bytes, const char* what) {
  if (!p) fail(SV_ERR_INVALID, std::string(what) + " is NULL");
  if ((uintptr_t)p % 16) fail(SV_ERR_INVALID, std::string(what) + " is not 16-byte aligned");
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(SV_ERR_INVALID, std::string(what) + " is not a CUDA pointer");
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    fail(SV_ERR_INVALID, std::string(what) + " is not device memory");
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (at.type == cudaMemoryTypeDevice && at.device != dev)
    fail(SV_ERR_INVALID, std::string(what) + " belongs to another device than the current one");
  if (AddrRangeFn fn = addr_range_fn()) {
    CUdeviceptr base = 0;
    size_t size = 0;
    if (fn(&base, &size, (CUdeviceptr)(uintptr_t)p) == CUDA_SUCCESS) {
      if ((uintptr_t)p + bytes > (uintptr_t)base + size)
        fail(SV_ERR_INVALID, std::string(what) + " is smaller than the requested size");
    }
  }
}

namespace {

// ----------------------------------------------------------- scratch per stream

struct Workspace {
  double* scratch = nullptr;
  size_t scratch_cap = 0;  // doubles
  double* out = nullptr;   // device results staged for host copies
  size_t out_cap = 0;      // doubles
  void* state = nullptr;   // sv_run_host state buffer
  size_t state_cap = 0;    // bytes
};

std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

void grow(void** p, size_t* cap, size_t want, cudaStream_t stream, const char* what) {
  if (*cap >= want) return;
  if (*p) {
    sync_stream(stream);
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
  }
  cudaError_t e = cudaMalloc(p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    fail(SV_ERR_OOM, std::string("cudaMalloc of ") + what + " failed: " + cudaGetErrorString(e));
  }
  *cap = want;
}

Workspace& workspace(cudaStream_t stream, size_t scratch_doubles, size_t out_doubles, size_t state_bytes) {
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_ws_mu);
  Workspace& w = g_ws[{dev, stream}];
  size_t sc = w.scratch_cap * sizeof(double), oc = w.out_cap * sizeof(double);
  grow((void**)&w.scratch, &sc, scratch_doubles * sizeof(double), stream, "reduction scratch");
  grow((void**)&w.out, &oc, std::max<size_t>(out_doubles, 64) * sizeof(double), stream, "result buffer");
  w.scratch_cap = sc / sizeof(double);
  w.out_cap = oc / sizeof(double);
  if (state_bytes) grow(&w.state, &w.state_cap, state_bytes, stream, "state buffer");
  return w;
}

std::map<std::tuple<int, cudaStream_t, std::string>, std::pair<void*, size_t>> g_named;

}  // namespace

void* scratch_buffer(cudaStream_t stream, const char* name, size_t bytes) {
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_ws_mu);
  auto& e = g_named[std::make_tuple(dev, stream, std::string(name))];
  grow(&e.first, &e.second, bytes < 256 ? 256 : bytes, stream, name);
  return e.first;
}

namespace {

// Pinned host staging per (device, stream, name), grow-only; `ready` is
// recorded after the last copy out of it, so a rewrite waits for that copy.
struct Pinned {
  void* p = nullptr;
  size_t cap = 0;
  cudaEvent_t ready = nullptr;
};
std::map<std::tuple<int, cudaStream_t, std::string>, Pinned> g_pinned;

Pinned& pinned_buffer(cudaStream_t stream, const char* name, size_t bytes) {
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_ws_mu);
  Pinned& pb = g_pinned[std::make_tuple(dev, stream, std::string(name))];
  if (!pb.ready) cuda_check(cudaEventCreateWithFlags(&pb.ready, cudaEventDisableTiming), "cudaEventCreate");
  cuda_check(cudaEventSynchronize(pb.ready), "cudaEventSynchronize");
  if (pb.cap < bytes) {
    if (pb.p) cudaFreeHost(pb.p);
    pb.p = nullptr;
    pb.cap = 0;
    cudaError_t e = cudaHostAlloc(&pb.p, bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(SV_ERR_OOM, std::string("cudaHostAlloc of ") + name + " failed");
    }
    pb.cap = bytes;
  }
  return pb;
}

// ----------------------------------------------------------- kernel timing

struct ProfRec {
  std::string family;
  cudaEvent_t e0, e1;
  double bytes;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;

}  // namespace

Prof::Prof(cudaStream_t s, const char* fam, double b) : stream(s), family(fam), bytes(b) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    e0 = e1 = nullptr;
    return;
  }
  cudaEventRecord(e0, stream);
}

void Prof::done() {
  if (!e0) return;
  cudaEventRecord(e1, stream);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.push_back({family, e0, e1, bytes});
  e0 = e1 = nullptr;
}

namespace {

// ----------------------------------------------------------- programs

#ifndef SV_ROT_SPLIT
#define SV_ROT_SPLIT 1
#endif
constexpr bool g_rot_split = SV_ROT_SPLIT != 0;  // register phases in rotation + phase-table form

// A 2x2 unitary U written as g * diag(1, ephi) * [[C, -S], [S, C]] * diag(1, elam)
// with C = |U00| and S = |U10| (C^2 + S^2 = 1, |g| = |ephi| = |elam| = 1): the
// Z-Y-Z Euler form of a one-qubit gate.  With C = cos(alpha), S = sin(alpha),
// alpha in [0, pi/2], the rotation is kept as the shear pair
// (tan(alpha/2), sin(alpha)) = (S / (1 + C), S), both in [0, 1].
struct RotSplit {
  cplx g = 1.0, ephi = 1.0, elam = 1.0;
  double t = 0.0, s = 0.0;
};

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
  r.t = S / (1.0 + C);
  r.s = S;
  return true;
}

// Converts one sweep of the plan into the kernel's program: each op gets local
// positions and control masks; consecutive ops whose moving qubits fit four
// register slots form one register phase; dense k >= 3 blocks and wide
// diagonals get a shared-memory phase of their own.
template <typename R>
void build_program(const Plan& plan, const Sweep& sw, SweepProgram<R>& P, int rq_override = 0) {
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
  std::vector<Tmp> ts(sw.ops.size());
  for (size_t oi = 0; oi < sw.ops.size(); oi++) {
    const LOp& op = plan.ops[sw.ops[oi]];
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
  int cur_first = -1, cur_n = 0;
  uint32_t cur_need = 0;
  for (int o = 0; o < (int)ts.size(); o++) {
    if (ts[o].smem) {
      if (cur_n) add_phase(PH_REG, cur_first, cur_n, cur_need);
      cur_n = 0;
      cur_need = 0;
      add_phase(PH_SMEM, o, 1, 0);
      continue;
    }
    if (cur_n && __builtin_popcount(cur_need | ts[o].need) <= rq && cur_n < 255) {
      cur_need |= ts[o].need;
      cur_n++;
    } else {
      if (cur_n) add_phase(PH_REG, cur_first, cur_n, cur_need);
      cur_first = o;
      cur_n = 1;
      cur_need = ts[o].need;
    }
  }
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
  // Per-slot products of a run of uncontrolled one-qubit gates [o, end).
  auto merge_run = [&](int o, int end, std::vector<cplx>& mats) {
    mats.assign(4 * rq, 0.0);
    for (int s2 = 0; s2 < rq; s2++) mats[4 * s2] = mats[4 * s2 + 3] = 1.0;
    uint32_t present = 0;
    for (; o < end; o++) {
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
        std::vector<cplx> mats;
        const uint32_t present = merge_run(o, end, mats);
        fin.push_back(kron_op(present, mats));
        o = end;
      } else {
        fin.push_back(ts[o]);
        o++;
      }
    }
  };
  auto emit_phase_rot = [&](int first, int nops) {
    const int NT = 1 << rq;
    std::vector<cplx> tab(NT, 1.0);
    cplx sc = 1.0;
    auto tab_dep = [&](uint32_t slots) {
      for (int j = 0; j < NT; j++)
        for (int s2 = 0; s2 < rq; s2++)
          if (((slots >> s2) & 1u) && tab[j] != tab[j ^ (1 << s2)]) return true;
      return false;
    };
    auto flush = [&]() {
      bool id = sc == cplx(1.0);
      for (const cplx& x : tab)
        if (x != cplx(1.0)) id = false;
      if (id) return;
      Tmp t = blank(OPK_PHASE);
      t.m.resize(NT);
      for (int j = 0; j < NT; j++) t.m[j] = tab[j] * sc;
      fin.push_back(t);
      tab.assign(NT, 1.0);
      sc = 1.0;
    };
    for (int o = first; o < first + nops;) {
      const Tmp& t = ts[o];
      const DevOp& d = t.d;
      if (u1_free(t)) {
        int end = o;
        while (end < first + nops && u1_free(ts[end])) end++;
        std::vector<cplx> mats;
        const uint32_t present = merge_run(o, end, mats);
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
          for (int j = 0; j < NT; j++)
            if ((j >> s2) & 1) tab[j] *= sp[s2].elam;
          sc *= sp[s2].g;
        }
        if (tab_dep(present)) flush();
        Tmp k = blank(OPK_KROT);
        k.d.rmask = (uint8_t)present;
        k.m.assign(rq, 0.0);
        for (int s2 = 0; s2 < rq; s2++)
          if ((present >> s2) & 1u) k.m[s2] = cplx(sp[s2].t, sp[s2].s);
        fin.push_back(k);
        for (int s2 = 0; s2 < rq; s2++) {
          if (!((present >> s2) & 1u)) continue;
          for (int j = 0; j < NT; j++)
            if ((j >> s2) & 1) tab[j] *= sp[s2].ephi;
        }
        continue;
      }
      if (d.kind == OPK_SIGN && d.tmask == 0 && d.xmask == 0) {  // on register slots only
        for (int j = 0; j < NT; j++)
          if (((uint32_t)j & d.rmask) == d.rval) tab[j] = -tab[j];
        o++;
        continue;
      }
      if (d.kind == OPK_DIAG && d.tmask == 0 && d.xmask == 0) {
        bool regs = true;
        for (int i = 0; i < d.k; i++)
          if (d.rs[i] == 0xFF) regs = false;
        if (regs) {
          for (int j = 0; j < NT; j++) {
            if (((uint32_t)j & d.rmask) != d.rval) continue;
            int idx = 0;
            for (int i = 0; i < d.k; i++) idx |= ((j >> d.rs[i]) & 1) << i;
            tab[j] *= t.m[idx];
          }
          o++;
          continue;
        }
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
  auto make_fin = [&](bool rot) {
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
          emit_phase_rot(first, nops);
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
    for (const Tmp& t : fin) ncoef += t.m.size();
    return (int)fin.size() <= kMaxOps && ncoef <= (size_t)SweepProgram<R>::kPool;
  };
  if (!make_fin(g_rot_split) && !make_fin(false)) fail(SV_ERR_INVALID, "internal: program too long");
  P.h.nops = (int)fin.size();

  int coef = 0;
  for (size_t oi = 0; oi < fin.size(); oi++) {
    fin[oi].d.coef = (uint32_t)coef;
    for (const cplx& v : fin[oi].m) {
      if (coef >= SweepProgram<R>::kPool) fail(SV_ERR_INVALID, "internal: coefficient pool overflow");
      P.coef[coef].re = (R)v.real();
      P.coef[coef].im = (R)v.imag();
      coef++;
    }
    P.ops[oi] = fin[oi].d;
  }
  for (int p = 0; p < nph; p++)
    if (P.ph[p].kind == PH_REG)
      for (int o = P.ph[p].first; o < P.ph[p].first + P.ph[p].nops; o++)
        if (P.ops[o].kind == OPK_SIGN) P.ops[o].coef = pattern(P.ops[o].rmask, P.ops[o].rval);
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
      std::fprintf(stderr, ")");
    }
    std::fprintf(stderr, "\n");
  }
}

template <typename R>
void run_plan(void* state, const Plan& plan, cudaStream_t stream) {
  if (sweep_timed_out())
    fail(SV_ERR_TIMEOUT, "an earlier pass gave up waiting (2 s) for its tile copies; its state is not valid");
  static thread_local std::unique_ptr<SweepProgram<R>> prog;
  if (!prog) prog.reset(new SweepProgram<R>());
  const double bytes = 2.0 * (double)sizeof(Cx<R>) * (double)(1ull << plan.n);  // read + write the state
  for (const Sweep& sw : plan.sweeps) {
    build_program<R>(plan, sw, *prog);
    Prof pr(stream, "sweep", bytes);
    cuda_check(launch_sweep<R>(reinterpret_cast<Cx<R>*>(state), *prog, stream), "sweep launch");
    pr.done();
  }
}

sv_exec_opts opts_of(const sv_exec_opts* o) {
  sv_exec_opts r;
  std::memset(&r, 0, sizeof(r));
  if (o) r = *o;
  return r;
}

sv_exec_opts fuse_opts(int fuse) {
  sv_exec_opts r = opts_of(nullptr);
  r.fuse_max_k = fuse;
  return r;
}

void apply_circuit(void* state, int n, sv_dtype dtype, const sv_gate* gates, size_t n_gates, const double* pv,
                   size_t npv, const sv_exec_opts& opts, cudaStream_t stream) {
  Plan plan = make_plan(n, dtype, gates, n_gates, pv, npv, opts);
  if (dtype == SV_C64)
    run_plan<float>(state, plan, stream);
  else
    run_plan<double>(state, plan, stream);
}

void expect_z_all_dev(const void* state, int n, sv_dtype dtype, double* out_dev, cudaStream_t stream) {
  Workspace& w = workspace(stream, expect_z_all_scratch_doubles(n), n + 1, 0);
  Prof pr(stream, "expect_z_all", (double)amp_bytes(dtype) * (double)(1ull << n));
  struct Done {
    Prof& p;
    ~Done() { p.done(); }
  } done_{pr};
  if (dtype == SV_C64)
    cuda_check(launch_expect_z_all<float>((const Cx<float>*)state, n, w.scratch, w.scratch_cap, out_dev, stream),
               "expect_z_all launch");
  else
    cuda_check(launch_expect_z_all<double>((const Cx<double>*)state, n, w.scratch, w.scratch_cap, out_dev, stream),
               "expect_z_all launch");
}

}  // namespace
}  // namespace sv

using namespace sv;

struct sv_state {
  void* ptr;
  int n;
  sv_dtype dtype;
  cudaStream_t stream;
  size_t bytes;
};

extern "C" {

int sv_version(void) { return 100; }

const char* sv_last_error(void) { return g_last_error.c_str(); }

sv_status sv_init_basis(void* state, int n_qubits, sv_dtype dtype, uint64_t basis_index, void* stream) {
  return guarded([&] {
    check_dtype_n(n_qubits, dtype);
    if (basis_index >= (1ull << n_qubits)) fail(SV_ERR_INVALID, "basis_index out of range");
    check_device_buffer(state, amp_bytes(dtype) << n_qubits, "state");
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SV_C64)
      cuda_check(launch_init_basis<float>((Cx<float>*)state, n_qubits, basis_index, s), "init launch");
    else
      cuda_check(launch_init_basis<double>((Cx<double>*)state, n_qubits, basis_index, s), "init launch");
  });
}

sv_status sv_apply_circuit(void* state, int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                           const double* param_values, size_t n_param_values, int fuse_max_k, void* stream) {
  return guarded([&] {
    check_dtype_n(n_qubits, dtype);
    check_device_buffer(state, amp_bytes(dtype) << n_qubits, "state");
    apply_circuit(state, n_qubits, dtype, gates, n_gates, param_values, n_param_values, fuse_opts(fuse_max_k),
                  (cudaStream_t)stream);
  });
}

sv_status sv_apply_circuit_ex(void* state, int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                              const double* param_values, size_t n_param_values, const sv_exec_opts* opts,
                              void* stream) {
  return guarded([&] {
    check_dtype_n(n_qubits, dtype);
    check_device_buffer(state, amp_bytes(dtype) << n_qubits, "state");
    apply_circuit(state, n_qubits, dtype, gates, n_gates, param_values, n_param_values, opts_of(opts),
                  (cudaStream_t)stream);
  });
}

sv_status sv_expect(const void* state, int n_qubits, sv_dtype dtype, const sv_pauli_term* terms, size_t n_terms,
                    double* out, int out_on_device, void* stream) {
  return guarded([&] {
    check_dtype_n(n_qubits, dtype);
    if (n_terms < 1 || n_terms > 4096) fail(SV_ERR_INVALID, "n_terms must be in 1..4096");
    if (!terms) fail(SV_ERR_INVALID, "terms is NULL");
    if (!out) fail(SV_ERR_INVALID, "out is NULL");
    const uint64_t all = (1ull << n_qubits) - 1ull;
    for (size_t j = 0; j < n_terms; j++)
      if ((terms[j].x_mask | terms[j].z_mask) & ~all)
        fail(SV_ERR_INVALID, "term " + std::to_string(j) + " names a qubit beyond n_qubits");
    check_device_buffer(state, amp_bytes(dtype) << n_qubits, "state");
    if (out_on_device) check_device_buffer(out, n_terms * sizeof(double), "out");
    cudaStream_t s = (cudaStream_t)stream;
    Workspace& w = workspace(s, expect_terms_scratch_doubles(n_qubits, (int)n_terms), n_terms, 0);
    double* dst = out_on_device ? out : w.out;
    Prof pr(s, "expect_terms", (double)amp_bytes(dtype) * (double)(1ull << n_qubits));
    if (dtype == SV_C64)
      cuda_check(launch_expect_terms<float>((const Cx<float>*)state, n_qubits, terms, (int)n_terms, w.scratch,
                                            w.scratch_cap, dst, s),
                 "expect launch");
    else
      cuda_check(launch_expect_terms<double>((const Cx<double>*)state, n_qubits, terms, (int)n_terms, w.scratch,
                                             w.scratch_cap, dst, s),
                 "expect launch");
    pr.done();
    if (!out_on_device) {
      cuda_check(cudaMemcpyAsync(out, w.out, n_terms * sizeof(double), cudaMemcpyDeviceToHost, s), "result copy");
      sync_stream(s);
    }
  });
}

sv_status sv_expect_z_all(const void* state, int n_qubits, sv_dtype dtype, double* out, int out_on_device,
                          void* stream) {
  return guarded([&] {
    check_dtype_n(n_qubits, dtype);
    if (!out) fail(SV_ERR_INVALID, "out is NULL");
    check_device_buffer(state, amp_bytes(dtype) << n_qubits, "state");
    if (out_on_device) check_device_buffer(out, (n_qubits + 1) * sizeof(double), "out");
    cudaStream_t s = (cudaStream_t)stream;
    if (out_on_device) {
      expect_z_all_dev(state, n_qubits, dtype, out, s);
    } else {
      Workspace& w = workspace(s, expect_z_all_scratch_doubles(n_qubits), n_qubits + 1, 0);
      expect_z_all_dev(state, n_qubits, dtype, w.out, s);
      cuda_check(cudaMemcpyAsync(out, w.out, (n_qubits + 1) * sizeof(double), cudaMemcpyDeviceToHost, s),
                 "result copy");
      sync_stream(s);
    }
  });
}

sv_status sv_plan_info(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates,
                       const double* param_values, size_t n_param_values, const sv_exec_opts* opts,
                       int* out_blocks, int* out_sweeps, int* block_starts) {
  return guarded([&] {
    Plan plan = make_plan(n_qubits, dtype, gates, n_gates, param_values, n_param_values, opts_of(opts));
    if (std::getenv("SV_DEBUG_PLAN")) {  // print the device programs (host only)
      std::unique_ptr<SweepProgram<float>> pf(new SweepProgram<float>());
      for (const Sweep& sw : plan.sweeps) build_program<float>(plan, sw, *pf);
    }
    int nb = (int)plan.block_starts.size() - 1;
    if (out_blocks) *out_blocks = nb;
    if (out_sweeps) *out_sweeps = (int)plan.sweeps.size();
    if (block_starts)
      for (size_t i = 0; i < plan.block_starts.size(); i++) block_starts[i] = plan.block_starts[i];
  });
}

sv_status sv_run_host(int n_qubits, sv_dtype dtype, const void* state_in, const sv_gate* gates, size_t n_gates,
                      const double* param_values, size_t n_param_values, int fuse_max_k, double* out_z,
                      void* state_out, void* stream) {
  return guarded([&] {
    check_dtype_n(n_qubits, dtype);
    if (!out_z) fail(SV_ERR_INVALID, "out_z is NULL");
    Plan plan = make_plan(n_qubits, dtype, gates, n_gates, param_values, n_param_values, fuse_opts(fuse_max_k));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = amp_bytes(dtype) << n_qubits;
    Workspace& w = workspace(s, expect_z_all_scratch_doubles(n_qubits), n_qubits + 1, bytes);
    if (state_in) {
      cuda_check(cudaMemcpyAsync(w.state, state_in, bytes, cudaMemcpyHostToDevice, s), "state upload");
    } else if (dtype == SV_C64) {
      cuda_check(launch_init_basis<float>((Cx<float>*)w.state, n_qubits, 0, s), "init launch");
    } else {
      cuda_check(launch_init_basis<double>((Cx<double>*)w.state, n_qubits, 0, s), "init launch");
    }
    if (dtype == SV_C64)
      run_plan<float>(w.state, plan, s);
    else
      run_plan<double>(w.state, plan, s);
    expect_z_all_dev(w.state, n_qubits, dtype, w.out, s);
    cuda_check(cudaMemcpyAsync(out_z, w.out, (n_qubits + 1) * sizeof(double), cudaMemcpyDeviceToHost, s),
               "result copy");
    if (state_out)
      cuda_check(cudaMemcpyAsync(state_out, w.state, bytes, cudaMemcpyDeviceToHost, s), "state download");
    sync_stream(s);
  });
}

sv_status sv_alloc(int n_qubits, sv_dtype dtype, void* stream, sv_handle* out) {
  return guarded([&] {
    check_dtype_n(n_qubits, dtype);
    if (!out) fail(SV_ERR_INVALID, "out is NULL");
    *out = nullptr;
    std::unique_ptr<sv_state> h(new sv_state{nullptr, n_qubits, dtype, (cudaStream_t)stream, amp_bytes(dtype) << n_qubits});
    cudaError_t e = cudaMalloc(&h->ptr, h->bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(SV_ERR_OOM, std::string("cudaMalloc of the state failed: ") + cudaGetErrorString(e));
    }
    cudaError_t le = dtype == SV_C64 ? launch_init_basis<float>((Cx<float>*)h->ptr, n_qubits, 0, h->stream)
                                     : launch_init_basis<double>((Cx<double>*)h->ptr, n_qubits, 0, h->stream);
    if (le != cudaSuccess) {
      cudaFree(h->ptr);
      cuda_check(le, "init launch");
    }
    *out = h.release();
  });
}

sv_status sv_free(sv_handle h) {
  return guarded([&] {
    if (!h) return;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    cudaFree(h->ptr);
    delete h;
    cuda_check(e, "cudaStreamSynchronize");
  });
}

void* sv_state_ptr(sv_handle h) { return h ? h->ptr : nullptr; }

sv_status sv_set_state(sv_handle h, const void* src, int src_is_device) {
  return guarded([&] {
    if (!h || !src) fail(SV_ERR_INVALID, "NULL handle or source");
    if (src_is_device) check_device_buffer(src, h->bytes, "src");
    cuda_check(cudaMemcpyAsync(h->ptr, src, h->bytes, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               h->stream),
               "state copy");
    sync_stream(h->stream);
  });
}

sv_status sv_get_state(sv_handle h, void* dst, int dst_is_device) {
  return guarded([&] {
    if (!h || !dst) fail(SV_ERR_INVALID, "NULL handle or destination");
    if (dst_is_device) check_device_buffer(dst, h->bytes, "dst");
    cuda_check(cudaMemcpyAsync(dst, h->ptr, h->bytes, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               h->stream),
               "state copy");
    sync_stream(h->stream);
  });
}

sv_status sv_profile_enable(int on) {
  return guarded([&] {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (on) {
      for (auto& r : g_prof) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
      }
      g_prof.clear();
    }
    g_prof_on = on != 0;
  });
}

sv_status sv_profile_read(sv_profile_entry* out, int max_entries, int* n_out, int reset) {
  return guarded([&] {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::vector<sv_profile_entry> agg;
    for (auto& r : g_prof) {
      cuda_check(cudaEventSynchronize(r.e1), "cudaEventSynchronize");
      float ms = 0.f;
      cuda_check(cudaEventElapsedTime(&ms, r.e0, r.e1), "cudaEventElapsedTime");
      sv_profile_entry* e = nullptr;
      for (auto& a : agg)
        if (r.family == a.name) e = &a;
      if (!e) {
        agg.push_back(sv_profile_entry{});
        e = &agg.back();
        std::strncpy(e->name, r.family.c_str(), sizeof(e->name) - 1);
      }
      e->launches++;
      e->total_ms += ms;
      e->bytes += r.bytes;
    }
    if (n_out) *n_out = (int)agg.size();
    for (int i = 0; i < (int)agg.size() && i < max_entries && out; i++) out[i] = agg[i];
    if (reset) {
      for (auto& r : g_prof) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
      }
      g_prof.clear();
    }
  });
}

}  // extern "C"

namespace sv {
namespace {
template <typename R>
void run_batch_small(int nreq, sv_dtype dtype, const int* nq, const sv_gate* const* gates, const size_t* ng,
                     double* out, int out_on_device, cudaStream_t stream) {
  std::vector<Plan> plans;
  plans.reserve(nreq);
  size_t nprog = 0;
  int max_n = 1;
  sv_exec_opts o;
  std::memset(&o, 0, sizeof(o));
  for (int b = 0; b < nreq; b++) {
    plans.push_back(make_plan(nq[b], dtype, gates[b], ng[b], nullptr, 0, o, nq[b]));
    nprog += plans.back().sweeps.size();
    max_n = std::max(max_n, nq[b]);
  }
  const size_t prog_bytes = sizeof(SweepProgram<R>) * nprog;
  const size_t idx_bytes = sizeof(int) * (2 * (size_t)nreq + 1);
  const size_t total = prog_bytes + idx_bytes;
  Pinned& pb = pinned_buffer(stream, "small_batch_staging", total);
  SweepProgram<R>* hp = reinterpret_cast<SweepProgram<R>*>(pb.p);
  int* hfirst = reinterpret_cast<int*>(reinterpret_cast<char*>(pb.p) + prog_bytes);
  int* hnq = hfirst + nreq + 1;
  size_t k = 0;
  for (int b = 0; b < nreq; b++) {
    hfirst[b] = (int)k;
    hnq[b] = nq[b];
    for (const Sweep& sw : plans[b].sweeps) build_program<R>(plans[b], sw, hp[k++], kRegQ);
  }
  hfirst[nreq] = (int)k;
  char* dbuf = (char*)scratch_buffer(stream, "small_batch_programs", total);
  cuda_check(cudaMemcpyAsync(dbuf, pb.p, total, cudaMemcpyHostToDevice, stream), "program upload");
  cuda_check(cudaEventRecord(pb.ready, stream), "cudaEventRecord");
  const SweepProgram<R>* dp = reinterpret_cast<const SweepProgram<R>*>(dbuf);
  const int* dfirst = reinterpret_cast<const int*>(dbuf + prog_bytes);
  const int* dnq = dfirst + nreq + 1;
  double* dout = out_on_device ? out : (double*)scratch_buffer(stream, "small_batch_out", sizeof(double) * nreq);
  Prof pr(stream, "small_batch", 0.0);
  cuda_check(launch_small_batch<R>(dp, dfirst, dnq, nreq, max_n, dout, stream), "small batch launch");
  pr.done();
  if (!out_on_device) {
    cuda_check(cudaMemcpyAsync(out, dout, sizeof(double) * nreq, cudaMemcpyDeviceToHost, stream), "result copy");
    sync_stream(stream);
  }
}
}  // namespace
}  // namespace sv

extern "C" {

sv_status sv_run_batch_small(int n_requests, sv_dtype dtype, const int* n_qubits, const sv_gate* const* gates,
                             const size_t* n_gates, double* out_sum_z, int out_on_device, void* stream) {
  return guarded([&] {
    if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_INVALID, "unknown dtype");
    if (n_requests < 1 || n_requests > 65535) fail(SV_ERR_INVALID, "n_requests must be in 1..65535");
    if (!n_qubits || !gates || !n_gates || !out_sum_z) fail(SV_ERR_INVALID, "NULL argument");
    for (int b = 0; b < n_requests; b++)
      if (n_qubits[b] < 1 || n_qubits[b] > SV_SMALL_MAX_QUBITS)
        fail(SV_ERR_INVALID, "request " + std::to_string(b) + ": n_qubits must be in 1..12 for the packed launch");
    if (out_on_device) check_device_buffer(out_sum_z, sizeof(double) * n_requests, "out_sum_z");
    if (dtype == SV_C64)
      run_batch_small<float>(n_requests, dtype, n_qubits, gates, n_gates, out_sum_z, out_on_device,
                             (cudaStream_t)stream);
    else
      run_batch_small<double>(n_requests, dtype, n_qubits, gates, n_gates, out_sum_z, out_on_device,
                              (cudaStream_t)stream);
  });
}

sv_status sv_release_scratch(void) {
  return guarded([&] {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if (g_ws.empty()) return;
    cuda_check(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    for (auto& kv : g_ws) {
      cudaFree(kv.second.scratch);
      cudaFree(kv.second.out);
      cudaFree(kv.second.state);
    }
    g_ws.clear();
    for (auto& kv : g_named) cudaFree(kv.second.first);
    g_named.clear();
    for (auto& kv : g_pinned) {
      if (kv.second.p) cudaFreeHost(kv.second.p);
      if (kv.second.ready) cudaEventDestroy(kv.second.ready);
    }
    g_pinned.clear();
  });
}

}  // extern "C"
