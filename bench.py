#!/usr/bin/env python
"""Benchmark of the state-vector hot path on GB300.

Default workload (the headline metric, one JSON line on stdout):
  30-qubit fused layered circuit, complex64: 20 layers of Haar-angle U3 on
  every qubit plus CZ on even then odd neighbour pairs (1180 gates), fused into
  <= 5-qubit blocks.  One step = |0..0> initialisation + the whole circuit +
  the per-qubit <Z> read-out, on a state (8 GiB) far larger than L2.

value = effective HBM GB/s = algorithmic bytes of the step's kernels (each pass
over the state reads and writes 2^n amplitudes; initialisation writes them once;
the read-out reads them once) / device time of the step, summed over ranks.
e2e = the same bytes over host wall time of one sv_run_host call per step
(gate records in, <Z_q> read-out back); e2e.with_state_download also copies
the final 8 GiB state to pinned host memory every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: replicas only (each rank simulates its own copy of the workload; no
collective on the data path).  --impl reference times the CPU oracle on the
host cores instead, on bounded samples of the same workload.
"""

from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gate-apply HBM GB/s (% peak) at 30q c64; adjoint grads/s; serving req/s + p99"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--layers", type=int, default=20)
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c64")
    ap.add_argument("--fuse", type=int, default=5)
    ap.add_argument("--block-mode", type=int, default=0)
    ap.add_argument("--ops-per-pass", type=int, default=0)
    ap.add_argument("--tile-qubits", type=int, default=0, help="0: the library's tile width")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-gates", type=int, default=0, help="oracle sample size (0 = auto)")
    ap.add_argument("--workload", choices=["gates", "adjoint", "serving", "precision", "latency", "sampling",
                                           "batchlayer", "checkpoint"], default="gates")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--seq-duration", type=float, default=10.0)
    ap.add_argument("--sweep-rates", type=str, default="25,50,100,200",
                    help="serving: extra sub-saturation rates (req/s), each run for --sweep-duration s")
    ap.add_argument("--sweep-duration", type=float, default=10.0)
    ap.add_argument("--serving-warmup-s", type=float, default=3.0,
                    help="serving: seconds of the arrival process served before the measured stream")
    ap.add_argument("--drain", type=float, default=30.0, help="serving: seconds after the last arrival before "
                                                              "unfinished requests are counted")
    ap.add_argument("--no-extras", action="store_true", help="gates workload: skip the adjoint, serving and "
                                                              "complex128 figures of the default line")
    return ap.parse_args()


def max_over_ranks(ms: float, ws: int, device) -> float:
    """The job's time for the timed steps: the slowest rank's (all-reduce
    MAX over the process group), then a barrier.  One rank: its own."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_rate(units_per_rank_step: float, steps: int, ws: int, ms: float) -> float:
    """Whole-job throughput: every rank processes its own replica of the
    workload (weak scaling), so the units of all ranks over the job's time."""
    return ws * steps * units_per_rank_step / (ms / 1e3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_indices):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for row in csv.reader(fh):
                if len(row) < 9:
                    continue
                try:
                    idx = int(row[0])
                except ValueError:
                    continue
                if gpu_indices is not None and idx not in gpu_indices:
                    continue
                try:
                    sm.append(float(row[1]))
                    smax.append(float(row[2]))
                except ValueError:
                    pass
                for nm, v in zip(names, row[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ reference arm (CPU oracle)

L2_BYTES = 129e6  # GB300 L2


def step_config(args, n, n_gates, nblocks, npasses, amp):
    """The workload's config dict, the same for both arms."""
    return {"workload": "fused_layered_u3_cz_%dq_%dlayers_%s" % (n, args.layers, args.dtype),
            "n_qubits": n, "layers": args.layers, "gates": n_gates, "fuse_max_k": args.fuse,
            "block_mode": args.block_mode, "fused_blocks": nblocks, "passes_per_step": npasses,
            "l2": ("inputs larger than L2 (state %.1f GiB)" if (2 ** n) * amp > L2_BYTES else
                   "state fits in L2 (%.1f GiB), not flushed") % ((2 ** n) * amp / 2 ** 30),
            "parallelism": "single"}


def step_bytes(n, npasses, amp):
    """The metric's bytes of one step: every pass reads and writes the state,
    plus the initialisation write and the read-out read."""
    return (2 * npasses + 2) * (2 ** n) * amp


def run_reference(args, ws, rank):
    """The oracle on the host cores, on the GPU arm's workload and metric: each
    step applies a bounded sample of the circuit's gates, and the value is the
    step's bytes (as the GPU arm counts them) times the fraction of the
    circuit's gates applied per second, i.e. the same effective GB/s a GPU
    run at the oracle's gate rate would report."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    import paper_2608_09733_gb300 as sv
    from paper_2608_09733_gb300 import build as _build
    from workloads import fused_layered_u3_cz
    n = args.n
    amp = 8 if args.dtype == "c64" else 16
    gates = fused_layered_u3_cz(n, args.layers, seed=0)
    # the plan's block and pass counts name the workload; the host planner
    # runs no kernel
    _build.build()
    sv.load()
    nblocks, npasses, _ = sv.sv_plan_info(n, sv.SV_C64 if args.dtype == "c64" else sv.SV_C128, sv.Gates(gates),
                                          fuse_max_k=args.fuse, block_mode=args.block_mode,
                                          ops_per_pass=args.ops_per_pass, tile_qubits=args.tile_qubits)
    sample = args.cpu_sample_gates or (4 if n >= 28 else 59)
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[0] = 1.0
    t_steps = []
    for s in range(args.warmup + args.steps):
        g = gates[(s * sample) % len(gates):][:sample]
        t0 = time.perf_counter()
        psi = _oracle_inplace(oracle, n, g, psi)
        t1 = time.perf_counter()
        if s >= args.warmup:
            t_steps.append(t1 - t0)
    t = sum(t_steps)
    gates_per_s = args.steps * sample / t
    value = gates_per_s * step_bytes(n, npasses, amp) / len(gates) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": step_config(args, n, len(gates), nblocks, npasses, amp),
            "gates_per_s": gates_per_s,
            "oracle_traffic_gbs": args.steps * sample * 2 * (2 ** n) * 16 / t / 1e9,
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": oracle.n_threads(), "kind": "oracle",
                             "sample": "%d consecutive gates of the %d-gate circuit per step on a %d-qubit "
                                       "complex128 state, one pass per gate; value = the step's bytes x the "
                                       "fraction of the circuit's gates applied per second" %
                                       (sample, len(gates), n)},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _oracle_inplace(oracle, n, gates, psi):
    import ctypes
    pk = oracle._Packed(gates, None)
    rc = oracle.lib().og_apply_circuit(psi.ctypes.data_as(ctypes.c_void_p), n, pk.arr, pk.n)
    assert rc == 0
    return psi


def cpu_baseline_sample(n, gates, sample_gates, bytes_per_step):
    """The oracle on the host cores: a bounded sample of the same workload,
    reported in the metric's unit (the step's bytes times the fraction of the
    circuit's gates applied per second)."""
    import numpy as np

    import oracle
    avail = _mem_available_gb()
    if avail is not None and avail < 2.5 * (2 ** n) * 16 / 1e9 + 4:
        return {"value": None, "unit": "GB/s", "cores": oracle.n_threads(), "kind": "oracle",
                "sample": "skipped: host has %.0f GB available, the %d-qubit complex128 oracle needs %.0f GB"
                          % (avail, n, (2 ** n) * 16 / 1e9)}
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[0] = 1.0
    _oracle_inplace(oracle, n, gates[:1], psi)  # touch pages, warm threads
    t0 = time.perf_counter()
    _oracle_inplace(oracle, n, gates[1:1 + sample_gates], psi)
    t = time.perf_counter() - t0
    gates_per_s = sample_gates / t
    return {"value": gates_per_s * bytes_per_step / len(gates) / 1e9, "unit": "GB/s", "cores": oracle.n_threads(),
            "kind": "oracle", "gates_per_s": gates_per_s,
            "oracle_traffic_gbs": sample_gates * 2 * (2 ** n) * 16 / t / 1e9,
            "sample": "gates 1..%d of the %d-gate circuit on a %d-qubit complex128 state, one pass per gate "
                      "(%.1f s); value = the step's bytes x the fraction of the circuit's gates applied per "
                      "second" % (sample_gates, len(gates), n, t)}


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return None


def read_traffic(kernel: str, stamp: str):
    """Per-launch DRAM traffic from the committed ncu summary, when it was taken
    on the current sources (the summary records the source stamp)."""
    path = os.path.join(ROOT, "profiles", "%s.md" % kernel)
    if not os.path.exists(path):
        return None
    tr, st = None, None
    with open(path) as fh:
        for line in fh:
            if line.startswith("traffic_bytes_per_launch_full_size:"):
                tr = float(line.split(":", 1)[1])
            if line.startswith("source_stamp:"):
                st = line.split(":", 1)[1].strip()
    return tr if (tr is not None and st == stamp) else None


# ------------------------------------------------------------------ other workloads

def bench_adjoint(args):
    """20-qubit hardware-efficient ansatz, 10 layers (400 parameters), H =
    sum Z_i Z_i+1 + 0.7 sum X_i, batch of 64 parameter vectors, complex64,
    checkpoints every 2 layers: full gradient vectors per second, batched vs
    one vector per call."""
    import torch
    import paper_2608_09733_gb300 as sv
    from workloads import hea_hamiltonian, hea_params, hea_ring
    n, layers, batch = 20, 10, args.batch
    gates = sv.Gates(hea_ring(n, layers))
    terms = sv.pauli_terms(hea_hamiltonian(n, 0.7))
    P = 2 * n * layers
    th = hea_params(batch, P, seed=0)
    ck = 2 * 3 * n
    for _ in range(args.warmup):
        sv.sv_adjoint_grad(n, sv.SV_C64, gates, th, terms, checkpoint_every=ck)
    sv.sv_profile_enable(True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sv.sv_adjoint_grad(n, sv.SV_C64, gates, th, terms, checkpoint_every=ck)
    t = time.perf_counter() - t0
    prof = sv.sv_profile_read(reset=True)
    sv.sv_profile_enable(False)
    # one vector per call (the plain path), a few rows
    rows = min(8, batch)
    for _ in range(2):  # its buffers, and the template's compiled kernels
        sv.sv_adjoint_grad(n, sv.SV_C64, gates, th[:1], terms, checkpoint_every=ck)
    t1 = time.perf_counter()
    for b in range(rows):
        sv.sv_adjoint_grad(n, sv.SV_C64, gates, th[b:b + 1], terms, checkpoint_every=ck)
    t1 = time.perf_counter() - t1
    peaks, src = measured_peaks()
    # the reverse pass: its compiled kernels once the template has run twice
    # (inside the warm-up), else the interpreting one
    fam = "batch_sweep_rev_jit" if "batch_sweep_rev_jit" in prof else "batch_sweep_rev"
    rev = prof.get(fam, {"bytes": 0, "total_ms": float("nan"), "launches": 0})
    gbs = rev["bytes"] / (rev["total_ms"] / 1e3) / 1e9 if rev["launches"] else None
    return ({
        "metric": "adjoint grads/s (20q HEA, 400 params, batch %d, c64)" % args.batch, "value": args.steps * batch / t,
        "unit": "grads/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "dtype": "c64", "data": "synthetic",
        "config": {"workload": "hea_adjoint_20q_10layers_batch%d_ckpt2layers" % batch},
        "one_vector_per_call_grads_per_s": rows / t1,
        "roofline": {"bound": "hbm", "kernel": ("k_batch_sweep_jit<reverse>" if fam.endswith("_jit") else
                                                "k_batch_sweep<reverse>"), "achieved": gbs,
                     "peak": float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)), "unit": "GB/s",
                     "frac": gbs / float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)) if gbs else None},
        "kernels": prof})


def serving_cpu_baseline(stream, served, budget_s=15.0):
    """The oracle on the host cores, one request after another, over the
    leading requests of the same stream (up to ~budget_s of CPU work, n <= 18
    so each fits the oracle quickly); also reports how far the served results
    of those requests are from the oracle's."""
    import numpy as np
    import oracle
    from workloads import serving_circuit
    done = {r.rid: r for r in served if r.result is not None}
    t0 = time.perf_counter()
    n_req, worst = 0, 0.0
    for rid, (_, n, depth, seed) in enumerate(stream):
        if n > 18:
            continue
        _, zsum = oracle.expect_z_all(oracle.run(n, serving_circuit(n, depth, seed)), n)
        n_req += 1
        if rid in done:
            worst = max(worst, abs(done[rid].result - zsum))
        if time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    return {"value": n_req / t, "unit": "req/s", "cores": oracle.n_threads(), "kind": "oracle",
            "sample": "the first %d requests with n <= 18 of the stream, one at a time (%.1f s)" % (n_req, t),
            "max_abs_diff_vs_served": worst}


def bench_serving(args):
    """Poisson arrivals (default 2000 req/s for 60 s) of layered U3 + CNOT
    ladder circuits, n uniform 8..26, depth 5..40, sum <Z_i> each, complex64,
    150 GB admission budget; against one request at a time, plus a sweep of
    sub-saturation rates."""
    import paper_2608_09733_gb300 as sv
    from paper_2608_09733_gb300.serving import Server, run_sequential
    from workloads import serving_stream
    stream = serving_stream(rate=args.rate, duration=args.duration, seed=0)
    # warm-up: the same arrival process (another seed) for a few seconds, so
    # that the serving family's pass structures have their compiled kernels
    # (shared by every circuit of a structure) before the measured stream, as
    # in a server that has been up for a while
    warm = serving_stream(rate=args.rate, duration=args.serving_warmup_s, seed=99)
    srv = Server(sv.SV_C64, budget_bytes=150e9)
    t_warm = time.perf_counter()
    srv.run(warm)
    t_warm = time.perf_counter() - t_warm
    stats, reqs = srv.run(stream, time_limit=args.duration + args.drain)
    seq_stream = [r for r in stream if r[0] < args.seq_duration]
    seq, _ = run_sequential(seq_stream, sv.SV_C64, time_limit=args.seq_duration + 30.0)
    sweep = []
    for rate in [float(x) for x in args.sweep_rates.split(",") if x.strip()]:
        st = serving_stream(rate=rate, duration=args.sweep_duration, seed=1)
        s_stats, _ = Server(sv.SV_C64, budget_bytes=150e9).run(st, time_limit=args.sweep_duration + args.drain)
        d = s_stats.as_dict()
        sweep.append({"rate": rate, **{k: d[k] for k in ("offered", "completed", "rejected", "unfinished",
                                                           "req_per_s", "p50_ms", "p99_ms")}})
    line = {
        "metric": "serving req/s + p99 (Poisson %.0f req/s, n 8-26, depth 5-40, c64)" % args.rate,
        "value": stats.req_per_s, "unit": "req/s", "n_gpus": 1, "higher_is_better": True, "dtype": "c64",
        "data": "synthetic", "config": {"workload": "serving_poisson_%.0fhz_%.0fs" % (args.rate, args.duration),
                                        "budget_gb": 150,
                                        "warm_up": "%.0f s of the same arrival process (seed 99) served first "
                                                   "(%.1f s wall)" % (args.serving_warmup_s, t_warm)},
        "served": stats.as_dict(), "sequential": seq.as_dict(), "rate_sweep": sweep}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = serving_cpu_baseline(stream, reqs, budget_s=getattr(args, "serving_cpu_s", 15.0))
    return line


def bench_precision(args):
    """24 qubits, 600 gates (400 Haar U(2) + 200 Haar SU(4) on random pairs,
    seeded shuffle), complex64 and complex128 on the GPU against the FP64
    oracle (timed as the CPU baseline of this workload): fidelity
    |<psi_oracle|psi>|^2 and max |psi - psi_oracle| after 100, 200 and 600
    gates."""
    import numpy as np
    import torch
    import oracle
    import paper_2608_09733_gb300 as sv
    from workloads import precision_sweep
    n = 24
    gates = precision_sweep(n, 400, 200, seed=0)
    cuts = (100, 200, 600)
    t0 = time.perf_counter()
    refs, psi = {}, None
    for a, b in zip((0,) + cuts[:-1], cuts):
        psi = oracle.run(n, gates[a:b], init=psi)
        refs[b] = psi.copy()
    t_oracle = time.perf_counter() - t0
    rows = []
    for dt, tdt in ((sv.SV_C64, torch.complex64), (sv.SV_C128, torch.complex128)):
        st = torch.empty(1 << n, dtype=tdt, device="cuda")
        sv.sv_init_basis(st, 0)
        done = 0
        for cut in cuts:
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sv.sv_apply_circuit(st, gates[done:cut], fuse_max_k=5)
            e1.record()
            torch.cuda.synchronize()
            done = cut
            got = st.cpu().numpy().astype(np.complex128)
            ref = refs[cut]
            rows.append({"dtype": "c64" if dt == sv.SV_C64 else "c128", "gates": cut,
                         "fidelity": float(abs(np.vdot(ref, got)) ** 2),
                         "max_abs_err": float(np.abs(got - ref).max()),
                         "rel_l2_err": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                         "segment_ms": e0.elapsed_time(e1)})
    print(json.dumps({
        "metric": "precision sweep: fidelity and max-abs error vs FP64 after 100/200/600 gates (24q)",
        "value": rows[2]["max_abs_err"], "unit": "max |psi - psi_fp64| (c64, 600 gates)", "n_gpus": 1,
        "higher_is_better": False, "dtype": "c64+c128", "data": "synthetic",
        "config": {"workload": "precision_sweep_24q_400u2_200su4", "fuse_max_k": 5}, "rows": rows,
        "cpu_baseline": {"value": t_oracle, "unit": "s for 600 gates", "cores": oracle.n_threads(), "kind": "oracle",
                         "sample": "the whole 600-gate circuit, complex128"}}), flush=True)


def bench_latency(args):
    """12 qubits, complex128, 10 layers of RY + RZ on every qubit and a CNOT
    ladder (350 gates): wall-clock microseconds per circuit (init + apply +
    <Z> read-out) on the device, one circuit after another on one stream, and
    per circuit when 1024 of them share one packed launch."""
    import torch
    import paper_2608_09733_gb300 as sv
    from workloads import layered_ry_rz_cnot
    n, reps = 12, 200
    g = sv.Gates(layered_ry_rz_cnot(n, 10, 0))
    st = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    out = torch.zeros(n + 1, dtype=torch.float64, device="cuda")

    def one():
        sv.sv_init_basis(st, 0)
        sv.sv_apply_circuit(st, g, fuse_max_k=5)
        sv.sv_expect_z_all(st, out=out)
    for _ in range(20):
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        one()
    torch.cuda.synchronize()
    seq_us = (time.perf_counter() - t0) / reps * 1e6
    nb = 1024
    res = torch.empty(nb, dtype=torch.float64, device="cuda")
    for _ in range(3):
        sv.sv_run_batch_small([n] * nb, [g] * nb, sv.SV_C128, out=res)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        sv.sv_run_batch_small([n] * nb, [g] * nb, sv.SV_C128, out=res)
    torch.cuda.synchronize()
    packed_us = (time.perf_counter() - t0) / (5 * nb) * 1e6
    print(json.dumps({
        "metric": "12q c128 layered circuit latency (350 gates)", "value": seq_us, "unit": "us per circuit",
        "n_gpus": 1, "higher_is_better": False, "dtype": "c128", "data": "synthetic",
        "config": {"workload": "layered_ry_rz_cnot_12q_10layers_c128", "fuse_max_k": 5},
        "packed_us_per_circuit": packed_us, "packed_batch": nb}), flush=True)


def bench_sampling(args):
    """Finite-shot measurement of the 30-qubit complex64 state of the fused
    layered circuit: 2^20 shots per step from seeded uniforms (shots/s), and
    the normalised probability vector (GB/s of state read)."""
    import numpy as np
    import torch
    import paper_2608_09733_gb300 as sv
    from workloads import fused_layered_u3_cz
    n, shots = args.n, 1 << 20
    st = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    sv.sv_init_basis(st, 0)
    sv.sv_apply_circuit(st, fused_layered_u3_cz(n, 4, 0), fuse_max_k=5)
    u = np.random.default_rng(0).random(shots)
    out = torch.empty(shots, dtype=torch.int64, device="cuda")
    for _ in range(args.warmup):
        sv.sv_sample(st, u, out=out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sv.sv_sample(st, u, out=out)
    torch.cuda.synchronize()
    t_s = (time.perf_counter() - t0) / args.steps
    p = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    sv.sv_probabilities(st, out=p)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        sv.sv_probabilities(st, out=p)
    e1.record()
    torch.cuda.synchronize()
    t_p = e0.elapsed_time(e1) / args.steps / 1e3
    print(json.dumps({
        "metric": "finite-shot sampling shots/s (%dq c64 state, 2^20 shots per call)" % n, "value": shots / t_s,
        "unit": "shots/s", "n_gpus": 1, "higher_is_better": True, "dtype": "c64", "data": "synthetic",
        "config": {"workload": "sample_%dq_c64_1M_shots" % n}, "ms_per_call": t_s * 1e3,
        "probabilities_ms": t_p * 1e3,
        "probabilities_gbs": ((8 + 8 + 8) << n) / t_p / 1e9}), flush=True)


def bench_batchlayer(args):
    """BatchLayer (angle encoding RY(x_q), then 4 layers of RY, RZ weights and
    a CNOT ring) on 16 qubits, complex64: a batch of 256 input rows through
    forward (per-qubit <Z>) and backward (one batched adjoint pass): rows per
    second for forward + backward."""
    import numpy as np
    import torch
    import paper_2608_09733_gb300 as sv
    from workloads import Gate
    n, layers, batch = 16, 4, 256
    gates, slot = [Gate("ry", [q], slots=[q]) for q in range(n)], n
    for _ in range(layers):
        for q in range(n):
            gates += [Gate("ry", [q], slots=[slot]), Gate("rz", [q], slots=[slot + 1])]
            slot += 2
        gates += [Gate("x", [(q + 1) % n], controls=[q]) for q in range(n)]
    layer = sv.BatchLayer(gates, n, n_data=n, n_weights=slot - n, dtype=sv.SV_C64).cuda()
    x = torch.tensor(np.random.default_rng(0).uniform(0, np.pi, size=(batch, n)), device="cuda",
                     requires_grad=True)
    target = torch.tensor(np.random.default_rng(1).normal(size=(batch, n)), device="cuda")

    def step():
        layer.zero_grad()
        x.grad = None
        loss = (layer(x) * target).sum()
        loss.backward()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    t = (time.perf_counter() - t0) / args.steps
    return {
        "metric": "BatchLayer rows/s, forward + backward (16q, 4 layers, batch 256, c64)", "value": batch / t,
        "unit": "rows/s", "n_gpus": 1, "higher_is_better": True, "dtype": "c64", "data": "synthetic",
        "config": {"workload": "batchlayer_16q_4layers_batch256", "parameters": slot,
                   "tensors": "inputs, weights, targets and gradients on the GPU (device-array entry points)"},
        "ms_per_step": t * 1e3}


def bench_checkpoint(args):
    """Adjoint checkpoint policies (Sec. 7.3) on a 24-qubit HEA, 10 layers,
    batch 4, complex64, a segment every 2 layers: time per gradient batch and
    the device memory the kept states take, for every state kept, 2 kept (the
    rest recomputed) and none kept."""
    import numpy as np
    import paper_2608_09733_gb300 as sv
    from workloads import hea_hamiltonian, hea_params, hea_ring
    n, layers, batch = 24, 10, 4
    gates, H = hea_ring(n, layers), hea_hamiltonian(n)
    P = 2 * n * layers
    params = hea_params(batch, P, seed=0)
    per_layer = 3 * n
    state_bytes = 8 * 2 ** n * batch
    segments = layers // 2
    rows, ref = [], None
    for stored in (-1, 2, 0):
        kw = dict(checkpoint_every=2 * per_layer, stored_states=stored)
        for _ in range(max(1, args.warmup)):
            sv.sv_adjoint_grad_ex(n, sv.SV_C64, gates, params, H, **kw)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, g = sv.sv_adjoint_grad_ex(n, sv.SV_C64, gates, params, H, **kw)
        t = (time.perf_counter() - t0) / args.steps
        ref = g if ref is None else ref
        kept = segments - 1 if stored < 0 else min(stored, segments - 1)
        rows.append({"stored_states": stored, "kept": kept, "kept_gb": kept * state_bytes / 1e9,
                     "ms_per_batch": t * 1e3, "grads_per_s": batch / t,
                     "max_grad_diff_vs_all_kept": float(np.abs(g - ref).max())})
    print(json.dumps({
        "metric": "adjoint checkpoint policies: time vs kept-state memory (24q HEA, 10 layers, batch 4, c64)",
        "value": rows[0]["grads_per_s"], "unit": "grads/s (all kept)", "n_gpus": 1, "higher_is_better": True,
        "dtype": "c64", "data": "synthetic", "config": {"workload": "hea_adjoint_24q_10layers_batch4_ckpt2layers"},
        "policies": rows}), flush=True)


# ------------------------------------------------------------------ figures beside the headline

def bench_c128_30q(args):
    """The same 30-qubit layered circuit on a complex128 state (16 GiB): per
    pass time against the FP64 pipe and HBM, whole-step time."""
    import torch
    import paper_2608_09733_gb300 as sv
    from workloads import fused_layered_u3_cz
    n = args.n
    glist = fused_layered_u3_cz(n, args.layers, seed=0)
    gates = sv.Gates(glist)
    _, npasses, _ = sv.sv_plan_info(n, sv.SV_C128, gates, fuse_max_k=args.fuse)
    st = torch.empty(2 ** n, dtype=torch.complex128, device="cuda")
    z = torch.empty(n + 1, dtype=torch.float64, device="cuda")

    def step():
        sv.sv_init_basis(st, 0)
        sv.sv_apply_circuit(st, gates, fuse_max_k=args.fuse)
        sv.sv_expect_z_all(st, out=z)
    step()
    torch.cuda.synchronize()
    sv.sv_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 2
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    prof = sv.sv_profile_read(reset=True)
    sv.sv_profile_enable(False)
    ms = e0.elapsed_time(e1) / steps
    sw = prof.get("sweep", {"launches": 0, "total_ms": float("nan"), "bytes": 0.0})
    per_pass = sw["total_ms"] / max(1, sw["launches"])
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    # FP64 work of the gates: 14 real flops per amplitude per U3 (a dense
    # 2x2 complex product), none for a CZ
    flops = sum(14.0 for g in glist if g.name == "u3") * (2 ** n)
    fp64 = flops * steps / (sw["total_ms"] / 1e3) / 1e12 if sw["launches"] else None
    del st
    torch.cuda.empty_cache()
    return {"metric": "30q c128 fused layered circuit", "value": ms, "unit": "ms per step", "dtype": "c128",
            "config": {"workload": "fused_layered_u3_cz_%dq_%dlayers_c128" % (n, args.layers),
                       "passes_per_step": npasses, "steps": steps},
            "ms_per_pass": per_pass,
            "hbm": {"achieved": 2 * (2 ** n) * 16 / (per_pass / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": 2 * (2 ** n) * 16 / (per_pass / 1e3) / 1e9 / hbm, "peak_source": src + " hbm_gbs"},
            "gate_flops": {"achieved": fp64, "unit": "TFLOP/s",
                           "note": "the U3s' dense 2x2 complex products (14 flops per amplitude) per second; the "
                                   "kernel runs them as scaled rotations and phase tables in fewer FP64 "
                                   "operations, so this is not an FP64-pipe utilisation"},
            "gates_per_s": len(glist) / (ms / 1e3)}


def run_extras(args):
    """The metric's other parts, each timed after the headline with its own
    clock record: adjoint gradients (20q HEA, batch 64), the serving stream
    (2000 req/s, bounded) with its sub-saturation sweep, and the 30-qubit
    circuit in complex128."""
    ex = {}
    jobs = [("adjoint", bench_adjoint, dict(batch=64, steps=5, warmup=3)),
            ("serving", bench_serving, dict(rate=2000.0, duration=10.0, seq_duration=5.0, sweep_duration=5.0,
                                            sweep_rates="25,50,100,200", drain=5.0, serving_cpu_s=5.0)),
            ("c128", bench_c128_30q, {})]
    for name, fn, over in jobs:
        a = argparse.Namespace(**vars(args))
        for k, v in over.items():
            setattr(a, k, v)
        clocks = ClockSampler()
        clocks.start()
        t0 = time.perf_counter()
        try:
            line = fn(a)
        except Exception as e:  # reported, never hides the headline
            line = {"error": repr(e)}
        line["wall_s"] = time.perf_counter() - t0
        line["clocks"] = clocks.stop(None)
        ex[name] = line
    return ex


# ------------------------------------------------------------------ our arm

def main():
    args = parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload != "gates":
        import torch
        torch.cuda.set_device(local)
        from paper_2608_09733_gb300 import build as _build
        _build.build()
        if rank == 0:
            fn = {"adjoint": bench_adjoint, "serving": bench_serving, "precision": bench_precision,
                  "latency": bench_latency, "sampling": bench_sampling, "batchlayer": bench_batchlayer,
                  "checkpoint": bench_checkpoint}[args.workload]
            clocks = ClockSampler()
            clocks.start()
            line = fn(args)
            if line is not None:
                line["clocks"] = clocks.stop(None)
                print(json.dumps(line), flush=True)
            else:
                clocks.stop(None)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2608_09733_gb300 import build as _build
    import paper_2608_09733_gb300 as sv
    from workloads import fused_layered_u3_cz

    _build.build()
    sv.load()
    stamp = _build.sweep_stamp()
    n, dt = args.n, (sv.SV_C64 if args.dtype == "c64" else sv.SV_C128)
    amp = 8 if dt == sv.SV_C64 else 16
    tdt = torch.complex64 if dt == sv.SV_C64 else torch.complex128
    gates = fused_layered_u3_cz(n, args.layers, seed=0)
    G = sv.Gates(gates)
    nblocks, npasses, _ = sv.sv_plan_info(n, dt, G, fuse_max_k=args.fuse, block_mode=args.block_mode,
                                          ops_per_pass=args.ops_per_pass, tile_qubits=args.tile_qubits)
    state = torch.empty(2 ** n, dtype=tdt, device="cuda")
    zout = torch.empty(n + 1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        sv.sv_init_basis(state, 0)
        sv.sv_apply_circuit_ex(state, G, None, fuse_max_k=args.fuse, block_mode=args.block_mode,
                               ops_per_pass=args.ops_per_pass, tile_qubits=args.tile_qubits)
        sv.sv_expect_z_all(state, out=zout)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler()
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sv.sv_profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    prof = sv.sv_profile_read(reset=True)
    sv.sv_profile_enable(False)
    ms = max_over_ranks(e0.elapsed_time(e1), ws, "cuda")
    clk = clocks.stop(None) if rank == 0 else None

    # the circuit's pass programs were compiled to their own kernels (by structure) on its
    # second run (a warm-up step); the timed steps launch those
    jit = sv.sv_jit_info()
    bytes_step = step_bytes(n, npasses, amp)  # passes r+w, init write, read-out read
    value = job_rate(bytes_step, args.steps, ws, ms) / 1e9
    gates_per_s = job_rate(len(gates), args.steps, ws, ms)
    peaks, peak_src = measured_peaks()
    # the dominant pass kernel: the program's own compiled kernel or the
    # interpreting TMA pass (complex64 states of 26 qubits and more), or the
    # cp.async one
    fams = [f for f in ("sweep_jit", "sweep_tma", "sweep") if f in prof]
    fam = max(fams, key=lambda f: prof[f]["total_ms"]) if fams else "sweep"
    kernel = "k_" + fam
    sw = prof.get(fam, {"launches": 0, "total_ms": float("nan"), "bytes": 0.0})
    launches = sum(v["launches"] for v in prof.values()) + args.steps  # + init kernel per step
    sweep_gbs = sw["bytes"] / (sw["total_ms"] / 1e3) / 1e9 if sw["launches"] else None
    peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    traffic = read_traffic("%s_%dq_%s" % (kernel, n, args.dtype), stamp)
    # ALU side: the complex arithmetic the gates need, 8 * 2^k - 2 real flops
    # per amplitude for a dense k-qubit gate (U3: 14), none for CZ; against
    # the FP32 (complex64) or FP64 (complex128) rate from unit counts x clock
    flops_step = sum(14.0 for g in gates if g.name == "u3") * (2 ** n)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = (152 * 128 * 2 * sm_mhz * 1e6 / 1e12) if dt == sv.SV_C64 else 1.25
    alu_achieved = flops_step * args.steps / (sw["total_ms"] / 1e3) / 1e12 if sw["launches"] else None

    # e2e: the same workload through the host-buffer entry point, one call per
    # step: the gate records in, |0..0> prepared, every pass, the <Z_q> read-out
    # copied back (the step's result); a second figure also downloads the
    # whole final state into pinned host memory every step
    e2e = None
    if not args.no_e2e:
        e2e_steps = max(1, min(args.steps, 3))

        def e2e_time(state_out):
            for _ in range(2):  # warm the buffers and the circuit's compiled pass kernels
                sv.sv_run_host(n, dt, G, fuse_max_k=args.fuse, state_out=state_out)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                z = sv.sv_run_host(n, dt, G, fuse_max_k=args.fuse, state_out=state_out)
            assert np.isfinite(z).all()
            return time.perf_counter() - t0

        te = e2e_time(None)
        e2e = {"value": ws * e2e_steps * bytes_step / te / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": len(gates) * 80, "d2h_bytes_per_step": 8 * (n + 1),
               "gates_per_s": ws * e2e_steps * len(gates) / te, "result": "<Z_q> of every qubit and their sum"}
        pinned = torch.empty(2 ** n, dtype=tdt).pin_memory()
        ts = e2e_time(pinned.numpy())
        e2e["with_state_download"] = {
            "value": ws * e2e_steps * bytes_step / ts / 1e9, "unit": "GB/s",
            "d2h_bytes_per_step": (2 ** n) * amp + 8 * (n + 1), "gates_per_s": ws * e2e_steps * len(gates) / ts,
            "download_gbs": (2 ** n) * amp / max(1e-9, (ts - te) / e2e_steps) / 1e9}
        del pinned
        sv.sv_release_scratch()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(n, gates, args.cpu_sample_gates or 24, bytes_step)

    extras = None
    if rank == 0 and ws == 1 and not args.no_extras and n == 30 and args.dtype == "c64":
        del state
        torch.cuda.empty_cache()
        extras = run_extras(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": dict(step_config(args, n, len(gates), nblocks, npasses, amp),
                           parallelism="replicas" if ws > 1 else "single"),
            "gates_per_s": gates_per_s,
            "pct_of_hbm_peak": 100.0 * value / ws / peak,
            "roofline": {"bound": "hbm", "kernel": kernel, "achieved": sweep_gbs, "peak": peak, "unit": "GB/s",
                         "frac": (sweep_gbs / peak) if sweep_gbs else None, "traffic": traffic,
                         "peak_source": peak_src + " hbm_gbs",
                         "launches": sw["launches"], "avg_launch_ms": sw["total_ms"] / max(1, sw["launches"]),
                         "alu_side": {"achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s",
                                      "frac": (alu_achieved / alu_peak) if alu_achieved else None,
                                      "peak_source": ("FP32: 152 SMs x 128 lanes x 2 x %.0f MHz" % sm_mhz)
                                      if dt == sv.SV_C64 else "FP64: nominal 1.25 TFLOP/s"}},
            "kernels": prof,
            "compiled_pass_kernels": {k: jit[k] for k in ("mode", "compiled", "failed", "compile_seconds")},
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        if extras is not None:
            line["adjoint"] = extras["adjoint"]
            line["serving"] = extras["serving"]
            line["c128"] = extras["c128"]
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
