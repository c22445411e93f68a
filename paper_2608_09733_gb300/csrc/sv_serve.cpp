// sv_serve.cpp -- serving sessions: a persistent packed kernel for small
// states fed from a work queue the host fills while it runs.
//
// The paper's NPU runs of small states were launch-bound (Sec. 9.3); the
// packed launch (sv_run_batch_small) removes most launches but still costs one
// launch, one program upload and one host wait per batch.  A session keeps one
// kernel resident instead: its CTAs take requests as the host publishes them
// (k_small_session in sv_sweep.cu), so a request costs its host planning, one
// program upload and a store of its queue entry.
//
// Host side of a session:
//   - pinned host memory mapped into the device holds the queue entries, the
//     published count (tail), the exit flag, the results and the done words;
//   - the device holds the programs (a ring arena), the claim counter (head)
//     and the status word;
//   - the kernel runs on a stream of its own (the device's highest priority)
//     and uploads go on another, both non-blocking, so they overlap;
//   - a ticket's slot (ticket mod capacity) and its arena range are reused
//     only once its done word is set.
// A session whose kernel has ended (its waits ran out while idle) is
// relaunched by the next submit; tickets published but not done are claimed
// again (a request done twice writes the same result).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <vector>

#include "sv_internal.h"

struct sv_small_session {
  sv_dtype dtype = SV_C64;
  int max_n = 12;
  int grid = 1;
  long long capacity = 0;
  int arena_programs = 0;
  double limit_s = 1.0;
  int device = 0;
  cudaStream_t run = nullptr, copy = nullptr;
  cudaEvent_t finished = nullptr;
  bool running = false;
  // mapped host memory
  sv::SmallEntry* entries = nullptr;
  long long* tail = nullptr;
  int* exit_flag = nullptr;
  double* results = nullptr;
  long long* done = nullptr;
  // device memory
  void* arena = nullptr;
  unsigned long long* head = nullptr;
  int* status = nullptr;
  // pinned staging for program uploads
  void* staging = nullptr;
  size_t staging_cap = 0;
  // bookkeeping
  long long next_ticket = 0;
  int arena_pos = 0;
  struct InFlight {
    long long ticket;
    int first, last;
  };
  std::deque<InFlight> inflight;  // in submission order
  std::mutex mu;
};

namespace sv {
namespace {

// Live sessions (for sessions_quiesce).
std::mutex g_sessions_mu;
std::vector<sv_small_session*> g_sessions;

size_t prog_bytes(sv_dtype d) { return d == SV_C64 ? sizeof(SweepProgram<float>) : sizeof(SweepProgram<double>); }

long long load_acquire(const long long* p) {
  return reinterpret_cast<const std::atomic<long long>*>(p)->load(std::memory_order_acquire);
}
void store_release(long long* p, long long v) {
  reinterpret_cast<std::atomic<long long>*>(p)->store(v, std::memory_order_release);
}

bool ticket_done(const sv_small_session* s, long long t) {
  return load_acquire(s->done + (t % s->capacity)) == t + 1;
}

// Drops finished tickets from the front of the in-flight list (their slots and
// arena ranges are free again).
void retire(sv_small_session* s) {
  while (!s->inflight.empty() && ticket_done(s, s->inflight.front().ticket)) s->inflight.pop_front();
}

void launch(sv_small_session* s) {
  SmallSessionDev d;
  d.entries = s->entries;
  d.tail = s->tail;
  d.exit_flag = s->exit_flag;
  d.head = s->head;
  d.results = s->results;
  d.done = s->done;
  d.status = s->status;
  d.capacity = s->capacity;
  d.limit_ns = (uint64_t)(s->limit_s * 1e9);
  cudaError_t e = s->dtype == SV_C64
                      ? launch_small_session<float>(d, (const SweepProgram<float>*)s->arena, s->max_n, s->grid, s->run)
                      : launch_small_session<double>(d, (const SweepProgram<double>*)s->arena, s->max_n, s->grid,
                                                     s->run);
  cuda_check(e, "session launch");
  cuda_check(cudaEventRecord(s->finished, s->run), "cudaEventRecord");
  s->running = true;
}

// Relaunches an ended kernel: claims restart at the oldest ticket not done.
void ensure_running(sv_small_session* s) {
  if (s->running) {
    const cudaError_t q = cudaEventQuery(s->finished);
    if (q == cudaErrorNotReady) return;
    cuda_check(q, "session kernel");
    s->running = false;
  }
  retire(s);
  const unsigned long long restart = s->inflight.empty() ? (unsigned long long)s->next_ticket
                                                         : (unsigned long long)s->inflight.front().ticket;
  cuda_check(cudaMemcpyAsync(s->head, &restart, sizeof(restart), cudaMemcpyHostToDevice, s->copy), "head reset");
  cuda_check(cudaStreamSynchronize(s->copy), "cudaStreamSynchronize");
  launch(s);
}

template <typename R>
void build_request_programs(int n, const sv_gate* gates, size_t ng, std::vector<SweepProgram<R>>& out) {
  // the lowering of sv_run_batch_small (no fusion blocks; every pass holds the
  // whole state), so the two give the same results bit for bit up to 12 qubits
  sv_exec_opts o;
  std::memset(&o, 0, sizeof(o));
  Plan plan = make_plan(n, sizeof(R) == 4 ? SV_C64 : SV_C128, gates, ng, nullptr, 0, o, n);
  // whole state in one tile: 16 amplitudes a thread up to 12 qubits, 32 at 13
  // and 14 (2^9 register groups: the session runs 512-thread CTAs for those)
  const int rq = n >= 13 ? 5 : kRegQ;
  const size_t k0 = out.size();
  out.resize(k0 + plan.sweeps.size());
  for (size_t i = 0; i < plan.sweeps.size(); i++) build_program<R>(plan, plan.sweeps[i], out[k0 + i], rq);
}

template <typename R>
void submit_batch(sv_small_session* s, int nreq, const int* nq, const sv_gate* const* gates, const size_t* ng,
                  int64_t* tickets) {
  std::vector<SweepProgram<R>> progs;
  std::vector<int> count(nreq);
  for (int b = 0; b < nreq; b++) {
    const size_t before = progs.size();
    build_request_programs<R>(nq[b], gates[b], ng[b], progs);
    count[b] = (int)(progs.size() - before);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  cuda_check(cudaSetDevice(s->device), "cudaSetDevice");
  retire(s);
  if ((long long)s->inflight.size() + nreq > s->capacity)
    fail(SV_ERR_OOM, "session full: " + std::to_string(s->inflight.size()) + " requests in flight of " +
                         std::to_string(s->capacity));
  // place the batch's programs contiguously in the arena ring, clear of the
  // programs of tickets still in flight
  const int total = (int)progs.size();
  if (total > s->arena_programs) fail(SV_ERR_OOM, "batch has more programs than the session's arena");
  int pos = s->arena_pos;
  if (pos + total > s->arena_programs) pos = 0;
  for (const auto& f : s->inflight) {
    const bool overlap = f.first < pos + total && pos < f.last;
    if (overlap) fail(SV_ERR_OOM, "session program arena full (requests in flight hold it)");
  }
  // uploads go through the fixed staging buffer in chunks: freeing and
  // growing pinned memory would synchronize the whole device, which waits for
  // the resident kernel
  const size_t per = sizeof(SweepProgram<R>), chunk = s->staging_cap / per;
  for (size_t done = 0; done < (size_t)total; done += chunk) {
    const size_t k = std::min(chunk, (size_t)total - done);
    std::memcpy(s->staging, progs.data() + done, per * k);
    cuda_check(cudaMemcpyAsync((char*)s->arena + per * ((size_t)pos + done), s->staging, per * k,
                               cudaMemcpyHostToDevice, s->copy),
               "program upload");
    cuda_check(cudaStreamSynchronize(s->copy), "cudaStreamSynchronize");
  }
  int first = pos;
  for (int b = 0; b < nreq; b++) {
    const long long t = s->next_ticket++;
    const long long slot = t % s->capacity;
    SmallEntry& e = s->entries[slot];
    e.first_prog = first;
    e.last_prog = first + count[b];
    e.n_qubits = nq[b];
    e.slot = (int32_t)slot;
    s->inflight.push_back({t, first, first + count[b]});
    first += count[b];
    tickets[b] = t;
  }
  s->arena_pos = pos + total;
  store_release(s->tail, s->next_ticket);  // entries before the count that publishes them
  ensure_running(s);
}

}  // namespace

// Loading a module waits for every resident kernel of the device to end, and
// a session's kernel stays resident until it idles past its wait limit: so a
// module load beside a live session would stall for that long (and a busy
// session never idles).  Quiesce takes each live session of the device (its
// lock held until release), sets its exit flag and waits for its kernel to
// end -- requests being simulated finish, claimed ones are claimed again
// later; release clears the flags and relaunches the sessions that have
// requests not done (the others relaunch on their next submit).
void sessions_quiesce(int device, std::vector<sv_small_session*>& held) {
  g_sessions_mu.lock();
  for (sv_small_session* s : g_sessions) {
    if (s->device != device) continue;
    s->mu.lock();
    held.push_back(s);
    if (!s->running) continue;
    reinterpret_cast<std::atomic<int>*>(s->exit_flag)->store(1, std::memory_order_release);
    cudaStreamSynchronize(s->run);
    s->running = false;
    reinterpret_cast<std::atomic<int>*>(s->exit_flag)->store(0, std::memory_order_release);
  }
}

void sessions_release(std::vector<sv_small_session*>& held) {
  for (sv_small_session* s : held) {
    retire(s);
    if (!s->inflight.empty()) {
      try {
        ensure_running(s);
      } catch (const Error&) {  // reported by the session's next call
      }
    }
    s->mu.unlock();
  }
  held.clear();
  g_sessions_mu.unlock();
}

namespace {

void free_session(sv_small_session* s) {
  if (s->entries) cudaFreeHost(s->entries);
  if (s->staging) cudaFreeHost(s->staging);
  if (s->arena) cudaFree(s->arena);
  if (s->head) cudaFree(s->head);
  if (s->run) cudaStreamDestroy(s->run);
  if (s->copy) cudaStreamDestroy(s->copy);
  if (s->finished) cudaEventDestroy(s->finished);
  delete s;
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_small_session_start(sv_dtype dtype, int capacity, int arena_programs, double wait_limit_s,
                                            int n_ctas, sv_small_session** out) {
  return guarded([&] {
    if (!out) fail(SV_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_INVALID, "unknown dtype");
    if (capacity < 1 || capacity > (1 << 20)) fail(SV_ERR_INVALID, "capacity must be in 1..2^20");
    if (arena_programs < 1 || arena_programs > (1 << 16)) fail(SV_ERR_INVALID, "arena_programs must be in 1..65536");
    if (!(wait_limit_s > 0.0 && wait_limit_s <= 3600.0)) fail(SV_ERR_INVALID, "wait_limit_s must be in (0, 3600]");
    std::unique_ptr<sv_small_session, void (*)(sv_small_session*)> s(new sv_small_session(), free_session);
    s->dtype = dtype;
    s->max_n = dtype == SV_C64 ? SV_SESSION_MAX_QUBITS : 12;
    s->capacity = capacity;
    s->arena_programs = arena_programs;
    s->limit_s = wait_limit_s;
    cuda_check(cudaGetDevice(&s->device), "cudaGetDevice");
    const int sms = device_sm_count();
    s->grid = n_ctas > 0 ? std::min(n_ctas, sms) : std::max(2, sms / 16);
    // The kernel's stream has the device's highest priority: a relaunch after
    // an idle exit queues behind the CTAs of whatever pass kernels other
    // streams have launched, and the block scheduler serves higher-priority
    // streams first as SMs free up.
    int least = 0, greatest = 0;
    cuda_check(cudaDeviceGetStreamPriorityRange(&least, &greatest), "cudaDeviceGetStreamPriorityRange");
    cuda_check(cudaStreamCreateWithPriority(&s->run, cudaStreamNonBlocking, greatest), "cudaStreamCreate");
    cuda_check(cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking), "cudaStreamCreate");
    cuda_check(cudaEventCreateWithFlags(&s->finished, cudaEventDisableTiming), "cudaEventCreate");
    // one mapped block: entries | tail | exit | results | done
    const size_t eb = sizeof(SmallEntry) * (size_t)capacity, rb = sizeof(double) * (size_t)capacity,
                 db = sizeof(long long) * (size_t)capacity;
    const size_t mapped = eb + 64 + rb + db;
    void* h = nullptr;
    cudaError_t e = cudaHostAlloc(&h, mapped, cudaHostAllocMapped);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(SV_ERR_OOM, "cudaHostAlloc of the session queue failed");
    }
    std::memset(h, 0, mapped);
    s->entries = (SmallEntry*)h;
    s->tail = (long long*)((char*)h + eb);
    s->exit_flag = (int*)((char*)h + eb + 8);
    s->results = (double*)((char*)h + eb + 64);
    s->done = (long long*)((char*)h + eb + 64 + rb);
    e = cudaMalloc(&s->arena, prog_bytes(dtype) * (size_t)arena_programs);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(SV_ERR_OOM, "cudaMalloc of the session program arena failed");
    }
    const size_t staging = prog_bytes(dtype) * (size_t)std::min(arena_programs, 256);
    e = cudaHostAlloc(&s->staging, staging, cudaHostAllocDefault);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(SV_ERR_OOM, "cudaHostAlloc of the session staging buffer failed");
    }
    s->staging_cap = staging;
    e = cudaMalloc(&s->head, 64);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(SV_ERR_OOM, "cudaMalloc of the session counters failed");
    }
    s->status = (int*)((char*)s->head + 16);
    cuda_check(cudaMemsetAsync(s->head, 0, 64, s->copy), "cudaMemset");
    cuda_check(cudaStreamSynchronize(s->copy), "cudaStreamSynchronize");
    launch(s.get());
    session_opened(s->device, s->grid);
    {
      std::lock_guard<std::mutex> lk(g_sessions_mu);
      g_sessions.push_back(s.get());
    }
    *out = s.release();
  });
}

extern "C" sv_status sv_small_session_submit(sv_small_session* s, int n_requests, const int* n_qubits,
                                             const sv_gate* const* gates, const size_t* n_gates, int64_t* tickets) {
  return guarded([&] {
    if (!s) fail(SV_ERR_INVALID, "session is NULL");
    if (n_requests < 1 || n_requests > 65535) fail(SV_ERR_INVALID, "n_requests must be in 1..65535");
    if (!n_qubits || !gates || !n_gates || !tickets) fail(SV_ERR_INVALID, "NULL argument");
    for (int b = 0; b < n_requests; b++)
      if (n_qubits[b] < 1 || n_qubits[b] > s->max_n)
        fail(SV_ERR_INVALID, "request " + std::to_string(b) + ": n_qubits must be in 1.." + std::to_string(s->max_n) +
                                 " for this session");
    if (s->dtype == SV_C64)
      submit_batch<float>(s, n_requests, n_qubits, gates, n_gates, tickets);
    else
      submit_batch<double>(s, n_requests, n_qubits, gates, n_gates, tickets);
  });
}

extern "C" sv_status sv_small_session_poll(sv_small_session* s, int64_t ticket, double* result, int* done) {
  return guarded([&] {
    if (!s || !result || !done) fail(SV_ERR_INVALID, "NULL argument");
    if (ticket < 0 || ticket >= s->next_ticket) fail(SV_ERR_INVALID, "unknown ticket");
    if (ticket + s->capacity < s->next_ticket) fail(SV_ERR_INVALID, "ticket's slot has been reused");
    *done = ticket_done(s, ticket) ? 1 : 0;
    *result = *done ? s->results[ticket % s->capacity] : 0.0;
  });
}

extern "C" sv_status sv_small_session_stop(sv_small_session* s) {
  int st = 0;
  const sv_status rc = guarded([&] {
    if (!s) fail(SV_ERR_INVALID, "session is NULL");
    {
      std::lock_guard<std::mutex> lk(g_sessions_mu);
      g_sessions.erase(std::remove(g_sessions.begin(), g_sessions.end(), s), g_sessions.end());
    }
    std::lock_guard<std::mutex> lk(s->mu);
    cuda_check(cudaSetDevice(s->device), "cudaSetDevice");
    reinterpret_cast<std::atomic<int>*>(s->exit_flag)->store(1, std::memory_order_release);
    cuda_check(cudaStreamSynchronize(s->run), "session kernel");
    cuda_check(cudaMemcpy(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
  });
  if (s) {
    session_closed(s->device, s->grid);
    free_session(s);
  }
  if (rc != SV_OK) return rc;
  if (st == SV_ERR_TIMEOUT) {
    set_last_error("a session CTA's wait for work ran out (the session was idle longer than its wait limit, or "
                   "its queue was never published); results of done tickets are valid");
    return SV_ERR_TIMEOUT;
  }
  return SV_OK;
}
