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
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "sv_hostcopy.h"
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

void sync_stream(cudaStream_t s) {
  cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  const int st = take_sweep_status(s);
  if (st == SV_ERR_TIMEOUT)
    fail(SV_ERR_TIMEOUT, "a pass kernel gave up waiting for its tile copies (bounded wait ran out); the state is not valid");
  if (st != SV_OK) fail(SV_ERR_CUDA, "reading the pass kernels' device status failed");
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
std::map<std::tuple<int, cudaStream_t, std::string>, Pinned> g_pinned;
}  // namespace

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

namespace {

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

// ----------------------------------------------------------- compiled circuits
//
// The pass programs of the last few circuits, keyed by the exact bytes of
// everything that decides them (n, precision, options, the gate records with
// their matrices, the parameter values).  A circuit applied again with the
// same inputs skips the host planning; every kernel still runs.

struct Compiled {
  std::vector<unsigned char> key;
  int n = 0;
  std::vector<SweepProgram<float>> pf;
  std::vector<SweepProgram<double>> pd;
  // the programs' structure keys (sv_jit.cpp), made on the first run
  mutable std::mutex jit_mu;
  mutable bool keys_made = false;
  mutable std::vector<std::string> keys;
};

constexpr size_t kCompiledMax = 8;                  // circuits kept
constexpr size_t kCompiledMaxPasses = 512;          // larger plans are not kept

std::mutex g_compiled_mu;
std::list<std::shared_ptr<const Compiled>> g_compiled;  // most recent first

std::vector<unsigned char> circuit_key(int n, sv_dtype dtype, const sv_gate* gates, size_t ng, const double* pv,
                                       size_t npv, const sv_exec_opts& opts) {
  std::vector<unsigned char> k;
  auto put = [&](const void* p, size_t b) {
    const unsigned char* c = (const unsigned char*)p;
    k.insert(k.end(), c, c + b);
  };
  const int32_t hdr[2] = {n, (int32_t)dtype};
  put(hdr, sizeof(hdr));
  put(&opts, sizeof(opts));
  put(&ng, sizeof(ng));
  put(&npv, sizeof(npv));
  for (size_t i = 0; i < ng; i++) {
    sv_gate g = gates[i];
    const double* m = g.matrix;
    g.matrix = nullptr;
    put(&g, sizeof(g));
    if (m && g.type == SV_GATE_UNITARY && g.n_targets >= 1 && g.n_targets <= 5)
      put(m, sizeof(double) * 2 * ((size_t)1 << (2 * g.n_targets)));
  }
  if (npv && pv) put(pv, sizeof(double) * npv);
  return k;
}

std::shared_ptr<const Compiled> compiled_circuit(int n, sv_dtype dtype, const sv_gate* gates, size_t ng,
                                                 const double* pv, size_t npv, const sv_exec_opts& opts) {
  std::vector<unsigned char> key = circuit_key(n, dtype, gates, ng, pv, npv, opts);
  {
    std::lock_guard<std::mutex> lk(g_compiled_mu);
    for (auto it = g_compiled.begin(); it != g_compiled.end(); ++it)
      if ((*it)->key == key) {
        std::shared_ptr<const Compiled> c = *it;
        g_compiled.erase(it);
        g_compiled.push_front(c);
        return c;
      }
  }
  Plan plan = make_plan(n, dtype, gates, ng, pv, npv, opts);
  auto c = std::make_shared<Compiled>();
  c->n = n;
  if (dtype == SV_C64) {
    c->pf.resize(plan.sweeps.size());
    for (size_t i = 0; i < plan.sweeps.size(); i++) build_program<float>(plan, plan.sweeps[i], c->pf[i]);
  } else {
    c->pd.resize(plan.sweeps.size());
    for (size_t i = 0; i < plan.sweeps.size(); i++) build_program<double>(plan, plan.sweeps[i], c->pd[i]);
  }
  if (plan.sweeps.size() <= kCompiledMaxPasses) {
    c->key = std::move(key);
    std::lock_guard<std::mutex> lk(g_compiled_mu);
    g_compiled.push_front(c);
    while (g_compiled.size() > kCompiledMax) g_compiled.pop_back();
  }
  return c;
}

template <typename R>
void run_programs(void* state, int n, const std::vector<SweepProgram<R>>& progs, cudaStream_t stream,
                  const std::vector<const JitKernel*>* jit = nullptr) {
  const double bytes = 2.0 * (double)sizeof(Cx<R>) * (double)(1ull << n);  // read + write the state
  for (size_t i = 0; i < progs.size(); i++) {
    Prof pr(stream, "sweep", bytes);
    const JitKernel* k = jit && i < jit->size() ? (*jit)[i] : nullptr;
    cuda_check(launch_sweep<R>(reinterpret_cast<Cx<R>*>(state), progs[i], stream, &pr.family, k), "sweep launch");
    pr.done();
  }
}

// The circuit's compiled pass kernels, by program structure: a structure is
// compiled (NVRTC, on the host) on its second use by any circuit (jit_mode()
// 1) or its first (2), and every later program of that structure -- this
// circuit run again, or another circuit of the same gates at other angles --
// launches the compiled kernel.  Until then the interpreting kernel runs.
std::vector<const JitKernel*> jit_kernels(const Compiled& c, sv_dtype dtype) {
  const int mode = jit_mode();
  if (mode == 0 || dtype != SV_C64) return {};
  {
    std::lock_guard<std::mutex> lk(c.jit_mu);
    if (!c.keys_made) {
      c.keys.resize(c.pf.size());
      for (size_t i = 0; i < c.pf.size(); i++) c.keys[i] = jit_program_key(c.pf[i]);
      c.keys_made = true;
    }
  }
  return jit_program_kernels(c.pf, c.keys, mode == 2 ? 1 : 2);
}

void run_compiled(void* state, const Compiled& c, sv_dtype dtype, cudaStream_t stream) {
  if (dtype == SV_C64) {
    const std::vector<const JitKernel*> k = jit_kernels(c, dtype);
    run_programs<float>(state, c.n, c.pf, stream, &k);
  } else {
    run_programs<double>(state, c.n, c.pd, stream);
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
  run_compiled(state, *compiled_circuit(n, dtype, gates, n_gates, pv, npv, opts), dtype, stream);
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
    std::shared_ptr<const Compiled> prog =
        compiled_circuit(n_qubits, dtype, gates, n_gates, param_values, n_param_values, fuse_opts(fuse_max_k));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = amp_bytes(dtype) << n_qubits;
    Workspace& w = workspace(s, expect_z_all_scratch_doubles(n_qubits), n_qubits + 1, bytes);
    if (state_in) {
      cuda_check(copy_state_host(w.state, state_in, bytes, false, s), "state upload");
    } else if (dtype == SV_C64) {
      cuda_check(launch_init_basis<float>((Cx<float>*)w.state, n_qubits, 0, s), "init launch");
    } else {
      cuda_check(launch_init_basis<double>((Cx<double>*)w.state, n_qubits, 0, s), "init launch");
    }
    run_compiled(w.state, *prog, dtype, s);
    expect_z_all_dev(w.state, n_qubits, dtype, w.out, s);
    cuda_check(cudaMemcpyAsync(out_z, w.out, (n_qubits + 1) * sizeof(double), cudaMemcpyDeviceToHost, s),
               "result copy");
    if (state_out)
      cuda_check(copy_state_host(state_out, w.state, bytes, true, s), "state download");
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
    cuda_check(src_is_device ? cudaMemcpyAsync(h->ptr, src, h->bytes, cudaMemcpyDeviceToDevice, h->stream)
                             : copy_state_host(h->ptr, src, h->bytes, false, h->stream),
               "state copy");
    sync_stream(h->stream);
  });
}

sv_status sv_get_state(sv_handle h, void* dst, int dst_is_device) {
  return guarded([&] {
    if (!h || !dst) fail(SV_ERR_INVALID, "NULL handle or destination");
    if (dst_is_device) check_device_buffer(dst, h->bytes, "dst");
    cuda_check(dst_is_device ? cudaMemcpyAsync(dst, h->ptr, h->bytes, cudaMemcpyDeviceToDevice, h->stream)
                             : copy_state_host(dst, h->ptr, h->bytes, true, h->stream),
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

sv_status sv_jit_set_mode(int mode) {
  return guarded([&] {
    if (mode < -1 || mode > 2) fail(SV_ERR_INVALID, "mode must be -1, 0, 1 or 2");
    jit_set_mode(mode);
  });
}

sv_status sv_jit_info(int* mode, int* available, long long* compiled, long long* failed, long long* launches,
                      double* compile_seconds, char* message, size_t message_cap) {
  return guarded([&] {
    std::string why, last;
    const bool av = jit_available(&why);
    jit_stats(compiled, failed, launches, compile_seconds, &last);
    if (mode) *mode = jit_mode();
    if (available) *available = av ? 1 : 0;
    if (message && message_cap) {
      const std::string& m = av ? last : why;
      const size_t k = std::min(m.size(), message_cap - 1);
      std::memcpy(message, m.data(), k);
      message[k] = '\0';
    }
  });
}

sv_status sv_jit_check(int n_qubits, sv_dtype dtype, const sv_gate* gates, size_t n_gates, const double* param_values,
                       size_t n_param_values, const sv_exec_opts* opts, int compile, int arch, int* n_sources,
                       int* n_compiled, char* text, size_t text_cap) {
  return guarded([&] {
    check_dtype_n(n_qubits, dtype);
    if (!n_sources || !n_compiled) fail(SV_ERR_INVALID, "NULL argument");
    if (compile && (arch < 100 || arch > 200)) fail(SV_ERR_INVALID, "arch must be a compute capability such as 103");
    if (compile && !jit_available(nullptr)) fail(SV_ERR_UNSUPPORTED, "the run-time compiler is not available");
    Plan plan = make_plan(n_qubits, dtype, gates, n_gates, param_values, n_param_values, opts_of(opts));
    std::string err, src;
    if (dtype == SV_C64) {
      std::vector<SweepProgram<float>> progs(plan.sweeps.size());
      for (size_t i = 0; i < plan.sweeps.size(); i++) build_program<float>(plan, plan.sweeps[i], progs[i]);
      jit_check_programs<float>(progs, compile != 0, arch, n_sources, n_compiled, &err, &src);
    } else {
      std::vector<SweepProgram<double>> progs(plan.sweeps.size());
      for (size_t i = 0; i < plan.sweeps.size(); i++) build_program<double>(plan, plan.sweeps[i], progs[i]);
      jit_check_programs<double>(progs, compile != 0, arch, n_sources, n_compiled, &err, &src);
    }
    if (text && text_cap) {
      const std::string& m = err.empty() ? src : err;
      const size_t k = std::min(m.size(), text_cap - 1);
      std::memcpy(text, m.data(), k);
      text[k] = '\0';
    }
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
