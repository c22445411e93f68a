"""GPU tests of the serving rows: the packed small-state launch and the
resident session kernel against the oracle, the session's bounded waits, and
the serving loop's results alone vs in the mix (complex64: 1e-4 on
sum_q <Z_q>)."""

import time

import numpy as np
import pytest

import oracle
from paper_2608_09733_gb300 import binding as B
from workloads import random_circuit, serving_circuit, serving_stream

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dt", [B.SV_C64, B.SV_C128])
def test_packed_small_batch_matches_oracle(svlib, cuda_dev, dt):
    ns = [1, 2, 3, 4, 5, 7, 8, 9, 10, 11, 12, 6, 12]
    sets = [random_circuit(n, 40, seed=200 + i, max_controls=min(2, n - 1) if n > 1 else 0,
                           max_unitary_k=min(4, n)) for i, n in enumerate(ns)]
    got = B.sv_run_batch_small(ns, sets, dt)
    tol = 1e-4 if dt == B.SV_C64 else 1e-10
    for n, g, v in zip(ns, sets, got):
        _, s = oracle.expect_z_all(oracle.run(n, g), n)
        assert abs(v - s) < tol, (n, v, s)


def test_packed_small_batch_result_independent_of_batch(svlib, cuda_dev):
    ns = [8, 12, 10, 9]
    sets = [serving_circuit(n, 7, seed=n) for n in ns]
    mix = B.sv_run_batch_small(ns, sets)
    for i in range(len(ns)):
        alone = B.sv_run_batch_small([ns[i]], [sets[i]])
        assert alone[0] == mix[i]


def _wait(session, tickets, limit=20.0):
    t0, out = time.time(), {}
    while len(out) < len(tickets):
        assert time.time() - t0 < limit, "session results overdue"
        for t in tickets:
            if t not in out:
                ok, v = session.poll(t)
                if ok:
                    out[t] = v
        time.sleep(0.001)
    return [out[t] for t in tickets]


@pytest.mark.parametrize("dt", [B.SV_C64, B.SV_C128])
def test_session_results_match_oracle_and_packed_launch(svlib, cuda_dev, dt):
    top = 14 if dt == B.SV_C64 else 12  # 14 qubits: the 512-thread session kernel
    ns = [1, 3, 5, 7, 8, 9, 10, 11, 12, top, 6, top, 2, 12]
    sets = [random_circuit(n, 40, seed=300 + i, max_controls=min(2, n - 1) if n > 1 else 0,
                           max_unitary_k=min(4, n)) for i, n in enumerate(ns)]
    sets += [serving_circuit(n, 9, seed=n) for n in (8, 12, top)]
    ns += [8, 12, top]
    tol = 1e-4 if dt == B.SV_C64 else 1e-10
    s = B.SmallSession(dt, capacity=64, wait_limit_s=10.0, n_ctas=3)
    try:
        got = _wait(s, s.submit(ns[:8], sets[:8]) + s.submit(ns[8:], sets[8:]))
    finally:
        s.stop()
    for n, g, v in zip(ns, sets, got):
        _, ref = oracle.expect_z_all(oracle.run(n, g), n)
        assert abs(v - ref) < tol, (n, v, ref)
    small = [i for i, n in enumerate(ns) if n <= 12]
    packed = B.sv_run_batch_small([ns[i] for i in small], [sets[i] for i in small], dt)
    assert all(got[i] == p for i, p in zip(small, packed))  # same programs, same order: same bits


def test_session_times_out_when_the_host_withholds_work(svlib, cuda_dev):
    """The host never publishes a request nor asks the session to end: every
    CTA's bounded wait runs out, records SV_ERR_TIMEOUT and returns, and the
    host reads that status at stop (the GPU stays usable)."""
    import torch
    s = B.SmallSession(B.SV_C64, capacity=8, wait_limit_s=0.2, n_ctas=2)
    time.sleep(0.8)
    with pytest.raises(B.SvError) as e:
        s.stop()
    assert e.value.status == 5  # SV_ERR_TIMEOUT
    x = torch.ones(4, device="cuda")
    assert float(x.sum()) == 4.0


def test_session_relaunches_after_an_idle_timeout(svlib, cuda_dev):
    s = B.SmallSession(B.SV_C64, capacity=16, wait_limit_s=0.2, n_ctas=2)
    try:
        time.sleep(0.6)  # the kernel ends idle; the next submit relaunches it
        sets = [serving_circuit(n, 5, seed=n) for n in (8, 9, 13)]
        got = _wait(s, s.submit([8, 9, 13], sets))
    finally:
        with pytest.raises(B.SvError):
            s.stop()  # the idle expiry is reported
    for n, g, v in zip((8, 9, 13), sets, got):
        _, ref = oracle.expect_z_all(oracle.run(n, g), n)
        assert abs(v - ref) < 1e-4


def test_session_rejects_bad_requests(svlib, cuda_dev):
    s = B.SmallSession(B.SV_C64, capacity=4, wait_limit_s=10.0, n_ctas=1)
    try:
        with pytest.raises(B.SvError):
            s.submit([15], [serving_circuit(15, 2, seed=1)])  # beyond 14 qubits
        with pytest.raises(B.SvError) as e:
            s.submit([8] * 5, [serving_circuit(8, 2, seed=k) for k in range(5)])  # more than its capacity
        assert e.value.status == 3  # SV_ERR_OOM
    finally:
        s.stop()


@pytest.mark.parametrize("mode", ["session", "packed"])
def test_serving_loop_results_alone_equal_in_the_mix(svlib, cuda_dev, mode):
    import torch
    from paper_2608_09733_gb300.serving import Server, request_gates, run_sequential
    stream = serving_stream(rate=4000.0, duration=0.05, n_lo=8, n_hi=17, d_lo=2, d_hi=6, seed=3)
    assert len(stream) > 50
    srv = Server(B.SV_C64, budget_bytes=2e9, workers=4, max_small_batch=64, small_mode=mode)
    stats, reqs = srv.run(stream)
    assert stats.failed == 0, [r.error for r in reqs if r.error]
    assert stats.completed == len(stream) and stats.rejected == 0
    assert stats.small > 0 and stats.large > 0
    seq, sreqs = run_sequential(stream, B.SV_C64)
    for r, q in zip(reqs, sreqs):
        assert abs(r.result - q.result) < 1e-4, (r.n, r.result, q.result)
    # a sample against the oracle
    for r in reqs[:: max(1, len(reqs) // 8)]:
        if r.n <= 14:
            g = serving_circuit(r.n, r.depth, r.seed)
            _, s = oracle.expect_z_all(oracle.run(r.n, g), r.n)
            assert abs(r.result - s) < 1e-4, (r.n, r.result, s)
    torch.cuda.synchronize()


def test_admission_rejects_states_beyond_the_budget(svlib, cuda_dev):
    from paper_2608_09733_gb300.serving import Server
    stream = [(0.0, 20, 2, 1), (0.0, 10, 2, 2)]
    srv = Server(B.SV_C64, budget_bytes=(1 << 19) * 8, workers=1)
    stats, reqs = srv.run(stream)
    assert reqs[0].path == "rejected" and reqs[1].result is not None
    assert stats.rejected == 1 and stats.completed == 1
