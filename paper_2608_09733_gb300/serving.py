"""Continuous-batching serving loop for circuit requests on one GPU.

Requests (arrival time, n qubits, depth, seed) each ask for sum_q <Z_q> of a
layered U3 + CNOT-ladder circuit.  The loop admits them as they arrive and
keeps many on the device at once:

* small requests (n <= SV_SMALL_MAX_QUBITS) are packed into one launch of
  ``sv_run_batch_small``: one CTA per request, the whole state in shared
  memory, so they never touch HBM and cost one launch per batch;
* large requests run on a pool of worker threads, each with its own CUDA
  stream and device state buffer: ``sv_init_basis`` + ``sv_apply_circuit`` +
  ``sv_expect_z_all``.  A request is admitted only while the states in flight
  fit the HBM budget (its 2^n amplitudes count against it until its result is
  read); the worker threads plan in the C library with the GIL released, so
  their work overlaps on the device.

Requests that arrive while the queue already holds ``max_queue`` are
rejected; a request larger than the whole budget is rejected at admission.
Latency is completion time minus arrival time on the host clock.

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
    peak_inflight_bytes: int = 0
    extra: Dict[str, float] = field(default_factory=dict)

    def as_dict(self):
        d = dict(self.__dict__)
        d.update(d.pop("extra"))
        return d


def _angles(n, depth, seed):
    from workloads import serving_angles  # input generator (seeded)
    return serving_angles(n, depth, seed)


def request_gates(r: Request):
    return B.layered_u3_cnot_gates(r.n, _angles(r.n, r.depth, r.seed))


class Server:
    """See the module docstring.  ``amp_bytes`` is 8 for complex64."""

    def __init__(self, dtype: int = B.SV_C64, budget_bytes: float = 150e9, workers: int = 6,
                 max_small_batch: int = 1024, max_queue: int = 20000, fuse_max_k: int = 5,
                 small_max_n: int = 12):
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
        self.small_max_n = min(small_max_n, 12)
        self._lock = threading.Condition()
        self._inflight = 0
        self._peak = 0

    # ------------------------------------------------------------ large path
    def _worker(self, q: "queue.Queue", t0: float, stop: threading.Event):
        torch = self.torch
        stream = torch.cuda.Stream()
        bufs: Dict[int, "torch.Tensor"] = {}
        zout = torch.zeros(64, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            while not stop.is_set():
                try:
                    r = q.get(timeout=0.005)
                except queue.Empty:
                    continue
                if r is None:
                    break
                need = (1 << r.n) * self.amp
                with self._lock:
                    while self._inflight + need > self.budget and not stop.is_set():
                        self._lock.wait(0.005)
                    self._inflight += need
                    self._peak = max(self._peak, self._inflight)
                try:
                    st = bufs.get(r.n)
                    if st is None:
                        st = torch.empty(1 << r.n, dtype=self.tdt, device="cuda")
                        bufs[r.n] = st
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
                    with self._lock:
                        self._inflight -= need
                        self._lock.notify_all()

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
        stats = ServeStats(offered=len(reqs))
        small_q: collections.deque = collections.deque()
        large_q: "queue.Queue" = queue.Queue()
        stop = threading.Event()
        t0 = time.perf_counter()
        threads = [threading.Thread(target=self._worker, args=(large_q, t0, stop), daemon=True)
                   for _ in range(self.workers)]
        for t in threads:
            t.start()
        small_stream = torch.cuda.Stream()
        inflight_small = []  # (event, requests, out tensor)
        admitted_large: List[Request] = []
        nxt = 0
        try:
            while True:
                now = time.perf_counter() - t0
                if time_limit is not None and now > time_limit:
                    break
                # arrivals
                while nxt < len(reqs) and reqs[nxt].arrival <= now:
                    r = reqs[nxt]
                    nxt += 1
                    if (1 << r.n) * self.amp > self.budget or len(small_q) + large_q.qsize() >= self.max_queue:
                        r.path = "rejected"
                        stats.rejected += 1
                        continue
                    if r.n <= self.small_max_n:
                        small_q.append(r)
                    else:
                        admitted_large.append(r)
                        large_q.put(r)
                # completed small batches
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
                # launch the next packed batch (at most two in flight)
                if small_q and len(inflight_small) < 2:
                    batch = [small_q.popleft() for _ in range(min(len(small_q), self.max_small_batch))]
                    out = torch.empty(len(batch), dtype=torch.float64, device="cuda")
                    B.sv_run_batch_small([r.n for r in batch], [request_gates(r) for r in batch], self.dtype,
                                         out=out, stream=small_stream)
                    ev = torch.cuda.Event()
                    ev.record(small_stream)
                    inflight_small.append((ev, batch, out))
                    stats.small_batches += 1
                # large completions are recorded by the workers
                if nxt == len(reqs) and not small_q and not inflight_small:
                    while admitted_large and admitted_large[-1].done is not None:
                        admitted_large.pop()
                    if all(r.done is not None for r in admitted_large):
                        break
                    time.sleep(0.0005)
                elif not small_q:
                    wait = reqs[nxt].arrival - now if nxt < len(reqs) else 0.0005
                    time.sleep(min(0.0005, max(0.0, wait)))
        finally:
            stop.set()
            for _ in threads:
                large_q.put(None)
            for t in threads:
                t.join(timeout=30)
            torch.cuda.synchronize()
        stats.failed = sum(1 for r in reqs if r.path == "failed")
        done = [r for r in reqs if r.done is not None and r.path != "failed"]
        stats.completed = len(done)
        stats.unfinished = stats.offered - stats.completed - stats.rejected - stats.failed
        stats.small = sum(1 for r in done if r.path == "small")
        stats.large = sum(1 for r in done if r.path == "large")
        stats.peak_inflight_bytes = int(self._peak)
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
    amp = 8 if dtype == B.SV_C64 else 16
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
    del amp
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
