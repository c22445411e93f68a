"""GPU checks of the pass kernels compiled at run time from one program.

A compiled kernel runs the same register and shared-memory op functions as
the interpreting TMA pass kernel, in the same order, with every dispatch
decision made when the source is generated; so on every circuit the two give
the same bits, and the oracle bounds both.  Tile width 12 forces the TMA pass
(and so the compiled kernels) on 21- to 24-qubit states, where the oracle
checks every amplitude; 24 and 26 qubits run the stage-refill path.
"""

import numpy as np
import pytest

import oracle
from paper_2608_09733_gb300 import binding as B
from workloads import fused_layered_u3_cz, random_circuit, serving_circuit

pytestmark = pytest.mark.gpu

TOL_C64 = 1e-5


def run(n, gates, mode, fuse=0, block_mode=0, tile=12, profile=False):
    """Final state (host complex64) with the compile mode set for this run;
    also the launches of compiled kernels it made and, with profile, the
    kernel families it ran."""
    import torch
    B.sv_jit_set_mode(mode)
    try:
        before = B.sv_jit_info()["launches"]
        st = torch.empty(2 ** n, dtype=torch.complex64, device="cuda")
        B.sv_init_basis(st, 0)
        if profile:
            B.sv_profile_enable(True)
        B.sv_apply_circuit_ex(st, gates, fuse_max_k=fuse, block_mode=block_mode, tile_qubits=tile)
        # the stream, not the device: a live serving session's kernel stays
        # resident, and a device-wide wait would wait for it
        torch.cuda.current_stream().synchronize()
        fam = B.sv_profile_read() if profile else None
        if profile:
            B.sv_profile_enable(False)
        launches = B.sv_jit_info()["launches"] - before
    finally:
        B.sv_jit_set_mode(-1)
    return st.cpu().numpy(), launches, fam


def same_bits(a, b):
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


def maxabs(a, ref):
    return float(np.max(np.abs(a.astype(np.complex128) - ref)))


def test_jit_available_on_gpu_box(svlib, cuda_dev):
    info = B.sv_jit_info()
    assert info["available"], info["message"]


@pytest.mark.parametrize("n", [22, 26])
def test_jit_layered_bitwise_equals_interpreter(svlib, cuda_dev, n):
    gates = fused_layered_u3_cz(n, 8, seed=40 + n)
    _, passes, _ = B.sv_plan_info(n, B.SV_C64, gates, fuse_max_k=5, tile_qubits=12)
    a, la, _ = run(n, gates, 0, fuse=5)
    b, lb, fam = run(n, gates, 2, fuse=5, profile=True)
    assert la == 0
    assert lb == passes, (lb, passes)
    assert "sweep_jit" in fam and fam["sweep_jit"]["launches"] == passes, fam
    assert same_bits(a, b)
    info = B.sv_jit_info()
    assert info["failed"] == 0, info["message"]


@pytest.mark.parametrize("n,ng", [(21, 160), (22, 160), (24, 100)])
def test_jit_random_circuits_all_families(svlib, cuda_dev, n, ng):
    """Every op kind of a pass program: rotations and phase tables, bit flips
    and swaps, dense and diagonal ops with controls inside and outside the
    tile, fused dense blocks in shared memory."""
    gates = random_circuit(n, ng, seed=900 + n, max_controls=3, max_unitary_k=5)
    ref = oracle.run(n, gates)
    for fuse, mode in ((0, 0), (5, 0), (5, 1)):
        _, passes, _ = B.sv_plan_info(n, B.SV_C64, gates, fuse_max_k=fuse, block_mode=mode, tile_qubits=12)
        a, _, _ = run(n, gates, 0, fuse=fuse, block_mode=mode)
        b, lb, _ = run(n, gates, 2, fuse=fuse, block_mode=mode)
        assert lb == passes, (fuse, mode, lb, passes)
        assert maxabs(b, ref) < TOL_C64, (fuse, mode, maxabs(b, ref))
        assert same_bits(a, b), (fuse, mode, maxabs(a.astype(np.complex128), b.astype(np.complex128)))


def test_jit_serving_circuit_21q_against_oracle(svlib, cuda_dev):
    n = 21
    gates = serving_circuit(n, 12, seed=17)
    ref = oracle.run(n, gates)
    got, launches, _ = run(n, gates, 2, fuse=5)
    assert launches > 0
    assert maxabs(got, ref) < TOL_C64, maxabs(got, ref)


def test_jit_second_run_default_mode(svlib, cuda_dev):
    """Mode 1 (the default): a program structure's first use interprets, its
    second compiles and launches the compiled kernel, with the same bits (a
    random circuit, whose passes share no structure with each other or with
    other tests' circuits)."""
    n = 23
    gates = random_circuit(n, 90, seed=2323, max_controls=2, max_unitary_k=2)
    _, passes, _ = B.sv_plan_info(n, B.SV_C64, gates, fuse_max_k=0, tile_qubits=12)
    a, la, _ = run(n, gates, 1)
    b, lb, _ = run(n, gates, 1)
    assert la == 0 and lb == passes, (la, lb, passes)
    assert same_bits(a, b)


def test_structure_shared_across_angles(svlib, cuda_dev):
    """Two circuits with the same gates at other angles share their passes'
    compiled kernels: after one run of the first, the second (a new circuit)
    runs compiled on its first run, bit for bit as interpreted and within the
    bar of the oracle."""
    n = 22
    g1 = fused_layered_u3_cz(n, 6, seed=501)
    g2 = fused_layered_u3_cz(n, 6, seed=502)  # same structure, other Haar angles
    _, passes, _ = B.sv_plan_info(n, B.SV_C64, g2, fuse_max_k=5, tile_qubits=12)
    run(n, g1, 1, fuse=5)
    b, lb, _ = run(n, g2, 1, fuse=5)
    assert lb == passes, (lb, passes)
    a, _, _ = run(n, g2, 0, fuse=5)
    assert same_bits(a, b)
    assert maxabs(b, oracle.run(n, g2)) < TOL_C64


def test_compiled_tma_pass_beside_a_live_session(svlib, cuda_dev):
    """While a serving session's kernel is resident the TMA pass (and its
    compiled kernels) runs on the SMs the session leaves free; results match
    the oracle and the session still serves."""
    n = 22
    gates = fused_layered_u3_cz(n, 6, seed=611)
    _, passes, _ = B.sv_plan_info(n, B.SV_C64, gates, fuse_max_k=5, tile_qubits=12)
    import time
    ses = B.SmallSession(B.SV_C64, capacity=64, wait_limit_s=10.0, n_ctas=9)
    sets = [serving_circuit(8, 5, 1), serving_circuit(10, 5, 2)]
    try:
        tickets = ses.submit([8, 10], sets)
        got, launches, fam = run(n, gates, 2, fuse=5, profile=True)
        assert launches == passes and fam["sweep_jit"]["launches"] == passes, fam
        res = []
        t0 = time.time()
        for tk in tickets:
            done, v = ses.poll(tk)
            while not done and time.time() - t0 < 20.0:
                time.sleep(0.001)
                done, v = ses.poll(tk)
            assert done
            res.append(v)
    finally:
        ses.stop()
    assert maxabs(got, oracle.run(n, gates)) < TOL_C64
    for nn, g, v in zip((8, 10), sets, res):
        _, ref = oracle.expect_z_all(oracle.run(nn, g), nn)
        assert abs(v - ref) < 1e-4


def test_jit_off_keeps_interpreter(svlib, cuda_dev):
    n = 22
    gates = fused_layered_u3_cz(n, 4, seed=78)
    _, l1, _ = run(n, gates, 0, fuse=5)
    _, l2, fam = run(n, gates, 0, fuse=5, profile=True)
    assert l1 == 0 and l2 == 0
    assert "sweep_jit" not in fam and "sweep_tma" in fam, fam


def test_default_tiles_compile_mid_size_states(svlib, cuda_dev):
    """With no tile width given, a 22-qubit complex64 state plans 12-qubit
    tiles while the compiled kernels are on, so its passes run on the TMA path
    and compile; the state matches the oracle."""
    import torch
    n = 22
    gates = fused_layered_u3_cz(n, 10, seed=44)
    B.sv_jit_set_mode(2)
    try:
        _, passes, _ = B.sv_plan_info(n, B.SV_C64, gates, fuse_max_k=5)
        assert passes == B.sv_plan_info(n, B.SV_C64, gates, fuse_max_k=5, tile_qubits=12)[1]
        before = B.sv_jit_info()["launches"]
        st = torch.empty(2 ** n, dtype=torch.complex64, device="cuda")
        B.sv_init_basis(st, 0)
        B.sv_apply_circuit(st, gates, fuse_max_k=5)
        torch.cuda.synchronize()
        assert B.sv_jit_info()["launches"] - before == passes
    finally:
        B.sv_jit_set_mode(-1)
    ref = oracle.run(n, gates)
    assert maxabs(st.cpu().numpy(), ref) < TOL_C64


def test_threads_compiling_one_structure_at_once(svlib, cuda_dev):
    """Four threads run circuits of one new structure at once (each its own
    state and stream), so they compile the same kernel sources concurrently:
    the first kernel loaded stays in the cache and every thread's passes run
    compiled, each state within the bar of the oracle."""
    import threading
    import torch
    n = 21
    circs = [fused_layered_u3_cz(n, 7, seed=7000 + i) for i in range(4)]  # same structure, other angles
    _, passes, _ = B.sv_plan_info(n, B.SV_C64, circs[0], fuse_max_k=5, tile_qubits=12)
    states = [torch.empty(2 ** n, dtype=torch.complex64, device="cuda") for _ in circs]
    errors = []
    barrier = threading.Barrier(len(circs))

    def work(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                B.sv_init_basis(states[i], 0, stream=s)
                barrier.wait()
                B.sv_apply_circuit_ex(states[i], circs[i], fuse_max_k=5, tile_qubits=12, stream=s)
                s.synchronize()
        except Exception as e:  # reported below
            errors.append(repr(e))

    B.sv_jit_set_mode(2)
    try:
        before = B.sv_jit_info()["launches"]
        th = [threading.Thread(target=work, args=(i,)) for i in range(len(circs))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        launches = B.sv_jit_info()["launches"] - before
    finally:
        B.sv_jit_set_mode(-1)
    assert not errors, errors
    assert launches == passes * len(circs), (launches, passes)
    for st, g in zip(states, circs):
        assert maxabs(st.cpu().numpy(), oracle.run(n, g)) < TOL_C64


def test_bench_circuit_30q_compiled_equals_interpreted(svlib, cuda_dev):
    """At the size and launch configuration the bench times (30 qubits,
    complex64, the 1180-gate layered circuit fused to k <= 5, 12-qubit tiles):
    every compiled pass, with its copy-outs and shared-memory layouts, gives
    the interpreting kernel's bits over the whole 2^30-amplitude state, and
    the state keeps its norm."""
    import torch
    n = 30
    gates = fused_layered_u3_cz(n, 20, seed=0)
    _, passes, _ = B.sv_plan_info(n, B.SV_C64, gates, fuse_max_k=5)
    states = []
    for mode in (0, 2):
        B.sv_jit_set_mode(mode)
        try:
            before = B.sv_jit_info()["launches"]
            st = torch.empty(2 ** n, dtype=torch.complex64, device="cuda")
            B.sv_init_basis(st, 0)
            B.sv_apply_circuit(st, gates, fuse_max_k=5)
            torch.cuda.current_stream().synchronize()
            launches = B.sv_jit_info()["launches"] - before
        finally:
            B.sv_jit_set_mode(-1)
        assert launches == (0 if mode == 0 else passes), (mode, launches, passes)
        states.append(st)
    a, b = (s.view(torch.int32) for s in states)
    assert torch.equal(a, b)
    norm = float(torch.linalg.vector_norm(states[1].view(torch.float32), dtype=torch.float64))
    assert abs(norm - 1.0) < 1e-4
