"""Continuous-batching serving loop for circuit requests on one GPU.

Requests (arrival time, n qubits, depth, seed) each ask for sum_q <Z_q> of a
layered U3 + CNOT-ladder circuit.  The loop admits them as they arrive and
keeps many on the device at once:

* small requests (n <= 14 for complex64, 12 for complex128) go to a serving
  session (``SmallSession``): one kernel stays resident on a few SMs and its
  CTAs take requests from a work queue in mapped host memory, each running a
  whole circuit on a state held in shared memory.  The loop submits the
  requests that arrived since its last turn in one batch and polls their done
  words; no request costs a kernel launch.  The session's CTAs end after
  ``session_wait_s`` without work (the next submit relaunches them), which
  also bounds how long a device-wide synchronization waits for them.  (``small_mode="packed"`` uses the
  one-launch-per-batch ``sv_run_batch_small`` instead, for n <= 12.)
* large requests are admitted against the HBM budget: an admitted request
  gets its own device state (2^n amplitudes) from a pool of the budget's size
  allocated when the run starts (``StatePool``); the state counts against the
  budget until its result has been read, and waits on the device for one of
  the worker threads.  Each worker has its own CUDA stream and runs
  ``sv_init_basis`` + ``sv_apply_circuit`` + ``sv_expect_z_all`` on it; the
  workers plan in the C library with the GIL released, so their work overlaps
  on the device.  A request that does not fit yet waits in the host queue.

Rejections, by cause: ``over_budget`` (one state larger than the pool's
largest block) and ``queue_full`` (the host queue already holds ``max_queue``
requests).  Latency is completion time minus arrival time on the host clock.
``peak_resident_bytes`` is the most device memory the admitted states held at
once.

The paper has no serving layer; its nearest parts are the batched state
(Sec. 4.1 BatchSV) and task parallelism across devices (Sec. 7.4).
"""

from __future__ import annotations

import collections
import queue
import threading
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import binding as B


@dataclass
class Request:
    rid: int
    arrival: float
    n: int
    depth: int
    seed: int
    done: Optional[float] = None
    result: Optional[float] = None
    path: str = ""
    error: Optional[str] = None
    state: object = None
    offset: int = -1
    ticket: int = -1


@dataclass
class ServeStats:
    offered: int = 0
    completed: int = 0
    failed: int = 0
    rejected: int = 0
    unfinished: int = 0
    wall_s: float = 0.0
    req_per_s: float = 0.0
    p50_ms: Optional[float] = None
    p99_ms: Optional[float] = None
    mean_ms: Optional[float] = None
    small: int = 0
    large: int = 0
    small_batches: int = 0
    peak_resident_bytes: int = 0
    rejected_by: Dict[str, int] = field(default_factory=dict)
    extra: Dict[str, float] = field(default_factory=dict)

    def as_dict(self):
        d = dict(self.__dict__)
        d.update(d.pop("extra"))
        return d


class StatePool:
    """Device memory for the admitted states, allocated once when a run starts
    and carved into power-of-two blocks (a buddy allocator), so admitting and
    releasing requests never calls the CUDA allocator mid-run: a cudaFree there
    synchronizes the device, which would wait for the resident session kernel.

    The budget is cut into root blocks (its binary decomposition, in units of
    ``min_bytes``, roots at most ``max_block``); a request takes the smallest
    free block that holds it, split in halves on the way down, and a released
    block merges with its free buddy within its root."""

    def __init__(self, budget_bytes: float, min_bytes: int = 1 << 16, max_block: int = 1 << 30, alloc=None):
        units = int(budget_bytes) // min_bytes
        self.min = min_bytes
        self.roots = []  # (base, size)
        base = 0
        size = max_block
        while units and size >= min_bytes:
            k = size // min_bytes
            while units >= k:
                self.roots.append((base, size))
                base += size
                units -= k
            size //= 2
        self.capacity = base
        self.free: Dict[int, set] = collections.defaultdict(set)
        for b, sz in self.roots:
            self.free[sz].add(b)
        self.used = 0
        self.peak = 0
        self.buf = alloc(self.capacity) if (alloc is not None and self.capacity) else None

    def _root(self, off):
        lo, hi = 0, len(self.roots) - 1
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if self.roots[mid][0] <= off:
                lo = mid
            else:
                hi = mid - 1
        return self.roots[lo]

    def block_size(self, nbytes: int) -> int:
        sz = self.min
        while sz < nbytes:
            sz *= 2
        return sz

    def alloc(self, nbytes: int) -> Optional[int]:
        """Offset of a free block of at least nbytes, or None."""
        want = self.block_size(nbytes)
        sz = want
        while sz not in self.free or not self.free[sz]:
            sz *= 2
            if sz > max((r[1] for r in self.roots), default=0):
                return None
        off = min(self.free[sz])
        self.free[sz].discard(off)
        while sz > want:  # split, keeping the low half
            sz //= 2
            self.free[sz].add(off + sz)
        self.used += want
        self.peak = max(self.peak, self.used)
        return off

    def release(self, off: int, nbytes: int):
        sz = self.block_size(nbytes)
        self.used -= sz
        base, rsz = self._root(off)
        while sz < rsz:
            buddy = base + ((off - base) ^ sz)
            if buddy not in self.free[sz]:
                break
            self.free[sz].discard(buddy)
            off = min(off, buddy)
            sz *= 2
        self.free[sz].add(off)


def _angles(n, depth, seed):
    from workloads import serving_angles  # input generator (seeded)
    return serving_angles(n, depth, seed)


def request_gates(r: Request):
    return B.layered_u3_cnot_gates(r.n, _angles(r.n, r.depth, r.seed))


class Server:
    """See the module docstring.  ``amp`` is 8 bytes for complex64."""

    def __init__(self, dtype: int = B.SV_C64, budget_bytes: float = 150e9, workers: int = 6,
                 max_small_batch: int = 256, max_queue: int = 20000, fuse_max_k: int = 5,
                 small_max_n: Optional[int] = None, small_mode: str = "session", session_wait_s: float = 0.05):
        import torch
        self.torch = torch
        self.dtype = dtype
        self.amp = 8 if dtype == B.SV_C64 else 16
        self.tdt = torch.complex64 if dtype == B.SV_C64 else torch.complex128
        self.budget = float(budget_bytes)
        self.workers = workers
        self.max_small_batch = max_small_batch
        self.max_queue = max_queue
        self.fuse = fuse_max_k
        self.small_mode = small_mode
        cap = (B.SV_SESSION_MAX_QUBITS if dtype == B.SV_C64 else 12) if small_mode == "session" else 12
        self.small_max_n = cap if small_max_n is None else min(small_max_n, cap)
        self.session_wait_s = session_wait_s
        self._lock = threading.Condition()
        self._resident = 0
        self._peak = 0

    # ------------------------------------------------------------ large path
    def _release(self, r: Request):
        need = (1 << r.n) * self.amp
        r.state = None
        with self._lock:
            self._pool.release(r.offset, need)
            self._resident -= need
            self._lock.notify_all()

    def _worker(self, q: "queue.Queue", t0: float, stop: threading.Event):
        torch = self.torch
        stream = torch.cuda.Stream()
        zout = torch.zeros(64, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            while not stop.is_set():
                try:
                    r = q.get(timeout=0.005)
                except queue.Empty:
                    continue
                if r is None:
                    break
                try:
                    st = r.state
                    g = request_gates(r)
                    B.sv_init_basis(st, 0, stream=stream)
                    B.sv_apply_circuit(st, g, fuse_max_k=self.fuse, stream=stream)
                    B.sv_expect_z_all(st, out=zout[: r.n + 1], stream=stream)
                    ev = torch.cuda.Event()
                    ev.record(stream)
                    while not ev.query():  # poll: the sleep releases the GIL to the other workers
                        time.sleep(0.0001)
                    r.result = float(zout[r.n].item())
                    r.done = time.perf_counter() - t0
                    r.path = "large"
                except Exception as e:  # reported per request; the worker keeps serving
                    r.error = repr(e)
                    r.path = "failed"
                    r.done = time.perf_counter() - t0
                finally:
                    self._release(r)

    # ------------------------------------------------------------ loop
    def run(self, stream, time_limit: Optional[float] = None, realtime: bool = True) -> (ServeStats, List[Request]):
        """Serves ``stream`` = [(arrival_s, n, depth, seed), ...] (sorted).
        With ``realtime`` requests become visible at their arrival times; else
        all are queued at t = 0 (saturation throughput).  The run stops at
        ``time_limit`` seconds (default: last arrival + 120 s); requests not
        finished by then count as unfinished."""
        if time_limit is None:
            time_limit = (max((a for a, _, _, _ in stream), default=0.0) if realtime else 0.0) + 120.0
        torch = self.torch
        reqs = [Request(i, float(a) if realtime else 0.0, int(n), int(d), int(s))
                for i, (a, n, d, s) in enumerate(stream)]
        stats = ServeStats(offered=len(reqs), rejected_by={"over_budget": 0, "queue_full": 0})
        self._pool = StatePool(self.budget, alloc=lambda nb: torch.empty(nb, dtype=torch.uint8, device="cuda"))
        host_q: collections.deque = collections.deque()  # large requests waiting for budget
        small_new: List[Request] = []                     # small requests not yet submitted
        small_live: List[Request] = []                    # submitted, not done
        work_q: "queue.Queue" = queue.Queue()
        stop = threading.Event()
        session = None
        if self.small_mode == "session":
            session = B.SmallSession(self.dtype, wait_limit_s=self.session_wait_s)
        t0 = time.perf_counter()
        threads = [threading.Thread(target=self._worker, args=(work_q, t0, stop), daemon=True)
                   for _ in range(self.workers)]
        for t in threads:
            t.start()
        small_stream = torch.cuda.Stream() if session is None else None
        inflight_small = []  # packed mode: (event, requests, out tensor)
        admitted: List[Request] = []
        nxt = 0

        def waiting():
            return len(host_q) + len(small_new)

        def admit(r):  # gives r its device state if the pool has room
            need = (1 << r.n) * self.amp
            with self._lock:
                off = self._pool.alloc(need)
                if off is None:
                    return False
                self._resident += need
                self._peak = max(self._peak, self._resident)
            r.offset = off
            r.state = self._pool.buf[off:off + need].view(self.tdt)
            admitted.append(r)
            work_q.put(r)
            return True

        try:
            while True:
                now = time.perf_counter() - t0
                if time_limit is not None and now > time_limit:
                    break
                # arrivals
                while nxt < len(reqs) and reqs[nxt].arrival <= now:
                    r = reqs[nxt]
                    nxt += 1
                    if self._pool.block_size((1 << r.n) * self.amp) > max((z for _, z in self._pool.roots),
                                                                          default=0):
                        r.path = "rejected"
                        stats.rejected_by["over_budget"] += 1
                    elif r.n > self.small_max_n and not host_q and admit(r):
                        pass
                    elif waiting() >= self.max_queue:
                        r.path = "rejected"
                        stats.rejected_by["queue_full"] += 1
                    elif r.n <= self.small_max_n:
                        small_new.append(r)
                    else:
                        host_q.append(r)
                # admission of the queued large requests, in arrival order
                while host_q and admit(host_q[0]):
                    host_q.popleft()
                # small requests
                if session is not None:
                    if small_new:
                        batch = small_new[: self.max_small_batch]
                        try:
                            tickets = session.submit([r.n for r in batch], [request_gates(r) for r in batch])
                        except B.SvError as e:
                            if e.status != 3:  # SV_ERR_OOM: the session is full, try again next turn
                                raise
                        else:
                            for r, t in zip(batch, tickets):
                                r.ticket = t
                            small_live.extend(batch)
                            del small_new[: len(batch)]
                            stats.small_batches += 1
                    if small_live:
                        tdone = time.perf_counter() - t0
                        keep = []
                        for r in small_live:
                            ok, v = session.poll(r.ticket)
                            if ok:
                                r.result, r.done, r.path = v, tdone, "small"
                            else:
                                keep.append(r)
                        small_live = keep
                else:
                    keep = []
                    for ev, rs, out in inflight_small:
                        if ev.query():
                            vals = out.cpu().numpy()
                            tdone = time.perf_counter() - t0
                            for r, v in zip(rs, vals):
                                r.result, r.done, r.path = float(v), tdone, "small"
                        else:
                            keep.append((ev, rs, out))
                    inflight_small = keep
                    if small_new and len(inflight_small) < 2:
                        batch = small_new[: self.max_small_batch]
                        del small_new[: len(batch)]
                        out = torch.empty(len(batch), dtype=torch.float64, device="cuda")
                        B.sv_run_batch_small([r.n for r in batch], [request_gates(r) for r in batch], self.dtype,
                                             out=out, stream=small_stream)
                        ev = torch.cuda.Event()
                        ev.record(small_stream)
                        inflight_small.append((ev, batch, out))
                        stats.small_batches += 1
                # finished?
                small_busy = small_new or small_live or inflight_small
                if nxt == len(reqs) and not host_q and not small_busy:
                    while admitted and admitted[-1].done is not None:
                        admitted.pop()
                    if all(r.done is not None for r in admitted):
                        break
                    time.sleep(0.0005)
                elif not small_busy:
                    wait = reqs[nxt].arrival - now if nxt < len(reqs) else 0.0005
                    time.sleep(min(0.0005, max(0.0, wait)))
        finally:
            stop.set()
            for _ in threads:
                work_q.put(None)
            for t in threads:
                t.join(timeout=30)
            if session is not None:
                try:
                    session.stop()
                except B.SvError as e:
                    if e.status != 5:  # SV_ERR_TIMEOUT: the session sat idle past its limit; results stand
                        raise
            torch.cuda.synchronize()
            for r in reqs:  # states of requests left in the queues
                if r.state is not None:
                    self._release(r)
            self._pool.buf = None
        stats.rejected = sum(stats.rejected_by.values())
        stats.failed = sum(1 for r in reqs if r.path == "failed")
        done = [r for r in reqs if r.done is not None and r.path != "failed"]
        stats.completed = len(done)
        stats.unfinished = stats.offered - stats.completed - stats.rejected - stats.failed
        stats.small = sum(1 for r in done if r.path == "small")
        stats.large = sum(1 for r in done if r.path == "large")
        stats.peak_resident_bytes = int(self._peak)
        if done:
            lat = np.array([r.done - r.arrival for r in done]) * 1e3
            last = max(r.done for r in done)
            stats.wall_s = last
            stats.req_per_s = len(done) / last if last > 0 else float("nan")
            stats.p50_ms = float(np.percentile(lat, 50))
            stats.p99_ms = float(np.percentile(lat, 99))
            stats.mean_ms = float(lat.mean())
        return stats, reqs


def run_sequential(stream, dtype: int = B.SV_C64, fuse_max_k: int = 5, time_limit: Optional[float] = None,
                   realtime: bool = True) -> (ServeStats, List[Request]):
    """Baseline: one request at a time, one circuit launch sequence after
    another on one stream (no packing, no overlap), same latency definition."""
    import torch
    tdt = torch.complex64 if dtype == B.SV_C64 else torch.complex128
    reqs = [Request(i, float(a) if realtime else 0.0, int(n), int(d), int(s))
            for i, (a, n, d, s) in enumerate(stream)]
    stats = ServeStats(offered=len(reqs))
    bufs = {}
    zout = torch.zeros(64, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    for r in reqs:
        now = time.perf_counter() - t0
        if time_limit is not None and now > time_limit:
            break
        if r.arrival > now:
            time.sleep(r.arrival - now)
        st = bufs.get(r.n)
        if st is None:
            st = torch.empty(1 << r.n, dtype=tdt, device="cuda")
            bufs[r.n] = st
        g = request_gates(r)
        B.sv_init_basis(st, 0)
        B.sv_apply_circuit(st, g, fuse_max_k=fuse_max_k)
        B.sv_expect_z_all(st, out=zout[: r.n + 1])
        r.result = float(zout[r.n].item())
        r.done = time.perf_counter() - t0
        r.path = "sequential"
    done = [r for r in reqs if r.done is not None]
    stats.completed = len(done)
    stats.unfinished = stats.offered - stats.completed
    if done:
        lat = np.array([r.done - r.arrival for r in done]) * 1e3
        last = max(r.done for r in done)
        stats.wall_s = last
        stats.req_per_s = len(done) / last
        stats.p50_ms = float(np.percentile(lat, 50))
        stats.p99_ms = float(np.percentile(lat, 99))
        stats.mean_ms = float(lat.mean())
    return stats, reqs
