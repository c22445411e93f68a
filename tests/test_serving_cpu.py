"""The serving loop's host logic on the CPU: admission against the HBM budget
(each admitted large request holds its own state until its result is read),
routing by size to the small-state session or the packed launch,
queue-limit and over-budget rejections by cause, and that every request is
accounted for.  The device calls are replaced by fakes that take time in
proportion to the state size (no GPU is touched)."""
import time

import pytest
import torch

from paper_2608_09733_gb300 import binding as B
from workloads import serving_stream


class _Stream:
    cuda_stream = 0


class _Event:
    def __init__(self, *a, **k):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def query(self):
        return time.perf_counter() - self.t > 0.0005


class _StreamCtx:
    def __init__(self, s):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


@pytest.fixture
def fake_device(monkeypatch):
    calls = {"small": 0, "large": 0}
    empty, zeros = torch.empty, torch.zeros

    def host_empty(*a, **k):
        k.pop("device", None)
        return empty(*a, **k)

    def host_zeros(*a, **k):
        k.pop("device", None)
        return zeros(*a, **k)

    def small(nq, sets, dtype=0, out=None, stream=None):
        calls["small"] += len(nq)
        out.copy_(torch.tensor([float(n) for n in nq], dtype=out.dtype))  # sum <Z_q> of |0..0> = n
        return out

    class FakeSession:
        """Tickets finish a little after submission; results as for |0..0>."""

        def __init__(self, dtype=0, capacity=16384, wait_limit_s=5.0, **k):
            self.t, self.res, self.stopped = [], [], False

        def submit(self, nq, sets):
            calls["small"] += len(nq)
            base = len(self.t)
            now = time.perf_counter()
            self.t += [now] * len(nq)
            self.res += [float(n) for n in nq]
            return list(range(base, base + len(nq)))

        def poll(self, ticket):
            ok = time.perf_counter() - self.t[ticket] > 0.0003
            return ok, (self.res[ticket] if ok else 0.0)

        def stop(self):
            self.stopped = True

    def apply(st, gates, *a, **k):
        calls["large"] += 1
        time.sleep(2e-4 * (st.numel() >> 13))

    def expect(st, out=None, stream=None):
        n = out.numel() - 1
        out[n] = float(n)
        return out

    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: _Stream())
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "stream", _StreamCtx)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch, "empty", host_empty)
    monkeypatch.setattr(torch, "zeros", host_zeros)
    monkeypatch.setattr(B, "sv_run_batch_small", small)
    monkeypatch.setattr(B, "SmallSession", FakeSession)
    monkeypatch.setattr(B, "sv_init_basis", lambda st, i=0, stream=None: None)
    monkeypatch.setattr(B, "sv_apply_circuit", apply)
    monkeypatch.setattr(B, "sv_expect_z_all", expect)
    return calls


@pytest.mark.parametrize("mode", ["session", "packed"])
def test_admission_routing_and_accounting(fake_device, mode):
    from paper_2608_09733_gb300.serving import Server
    stream = serving_stream(rate=3000.0, duration=0.05, n_lo=8, n_hi=19, d_lo=2, d_hi=6, seed=3)
    budget = 8 * (1 << 18) * 3  # three 18-qubit complex64 states; 19-qubit requests exceed it
    srv = Server(B.SV_C64, budget_bytes=budget, workers=4, max_small_batch=64, small_mode=mode)
    stats, reqs = srv.run(stream, time_limit=30.0)
    assert stats.offered == len(stream)
    assert stats.completed + stats.rejected + stats.failed + stats.unfinished == stats.offered
    assert stats.failed == 0 and stats.unfinished == 0
    assert 0 < stats.peak_resident_bytes <= budget
    assert srv._resident == 0  # every admitted state was released
    n19 = sum(1 for r in reqs if 8 * (1 << r.n) > budget)
    assert stats.rejected_by == {"over_budget": n19, "queue_full": 0} and stats.rejected == n19
    assert srv.small_max_n == (14 if mode == "session" else 12)
    for r in reqs:
        if 8 * (1 << r.n) > budget:
            assert r.path == "rejected"
        else:
            assert r.path == ("small" if r.n <= srv.small_max_n else "large")
            assert r.result == float(r.n)  # the fake's sum <Z_q> for |0..0>
            assert r.done >= r.arrival and r.state is None
    assert fake_device["small"] == stats.small and fake_device["large"] == stats.large
    assert stats.small > 0 and stats.large > 0


def test_budget_holds_the_resident_states(fake_device):
    """With a burst of large requests the admitted states fill the budget and
    no further request is admitted until one is released."""
    from paper_2608_09733_gb300.serving import Server
    stream = [(0.0, 16, 2, i) for i in range(40)]
    budget = 8 * (1 << 16) * 5  # five 16-qubit states at once
    srv = Server(B.SV_C64, budget_bytes=budget, workers=2)
    stats, reqs = srv.run(stream, time_limit=30.0)
    assert stats.completed == 40 and stats.rejected == 0
    assert stats.peak_resident_bytes == budget  # the budget, not the worker count, bounds residency
    assert srv._resident == 0


def test_queue_limit_rejects(fake_device):
    from paper_2608_09733_gb300.serving import Server
    stream = serving_stream(rate=20000.0, duration=0.02, n_lo=16, n_hi=17, d_lo=2, d_hi=3, seed=4)
    srv = Server(B.SV_C64, budget_bytes=8 * (1 << 17) * 2, workers=1, max_queue=5)
    stats, _ = srv.run(stream, time_limit=30.0)
    assert stats.rejected_by["queue_full"] > 0 and stats.rejected_by["over_budget"] == 0
    assert stats.completed + stats.rejected == stats.offered


def test_state_pool_buddy_allocator():
    """Blocks never overlap, stay inside the pool, merge back to the roots
    when everything is released, and the budget's binary decomposition is
    what the pool holds."""
    import random
    from paper_2608_09733_gb300.serving import StatePool
    pool = StatePool(5 * (1 << 20) + 3 * (1 << 16), min_bytes=1 << 16, max_block=1 << 21)
    assert pool.capacity == 5 * (1 << 20) + 3 * (1 << 16)
    assert all(sz <= (1 << 21) for _, sz in pool.roots)
    rng = random.Random(7)
    live = {}
    for step in range(3000):
        if live and (rng.random() < 0.45 or len(live) > 40):
            off = rng.choice(list(live))
            pool.release(off, live.pop(off))
        else:
            nb = rng.choice([1 << 16, 1 << 17, 3 << 16, 1 << 19, 1 << 20, 1 << 21, 1 << 22])
            off = pool.alloc(nb)
            if off is None:
                continue
            sz = pool.block_size(nb)
            assert off % sz == 0 or any(b <= off < b + z and (off - b) % sz == 0 for b, z in pool.roots)
            assert 0 <= off and off + sz <= pool.capacity
            for o, n2 in live.items():
                s2 = pool.block_size(n2)
                assert off + sz <= o or o + s2 <= off, "overlap"
            live[off] = nb
        assert pool.used == sum(pool.block_size(v) for v in live.values()) <= pool.capacity
    for off, nb in list(live.items()):
        pool.release(off, nb)
    assert pool.used == 0
    assert sorted((b, z) for z, offs in pool.free.items() for b in offs) == sorted(pool.roots)
    assert pool.alloc(1 << 22) is None  # larger than the largest root
