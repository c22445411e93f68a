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
        torch.cuda.synchronize()
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
    """Mode 1 (the default): the first run of a circuit interprets, the
    second compiles and launches the compiled kernels, with the same bits."""
    n = 24
    gates = fused_layered_u3_cz(n, 5, seed=77)
    _, passes, _ = B.sv_plan_info(n, B.SV_C64, gates, fuse_max_k=5, tile_qubits=12)
    a, la, _ = run(n, gates, 1, fuse=5)
    b, lb, _ = run(n, gates, 1, fuse=5)
    assert la == 0 and lb == passes, (la, lb, passes)
    assert same_bits(a, b)


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
