"""CPU checks of the C-ABI library: it loads, exports every symbol that
include/sv.h declares, plans exactly the paper's fusion blocks, and rejects
bad input at the boundary -- all without touching a GPU."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2608_09733_gb300 import binding as B
from workloads import (Gate, fused_layered_u3_cz, hea_ring, layered_ry_rz_cnot, precision_sweep,
                       random_circuit)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sv_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(svlib):
    decl = declared_symbols()
    assert len(decl) >= 10
    assert sorted(B.EXPORTS) == decl
    for name in decl:
        assert hasattr(svlib, name), name
    assert B.sv_version() == 100


@pytest.mark.parametrize("kmax", [2, 3, 4, 5])
@pytest.mark.parametrize("seed", range(3))
def test_fusion_blocks_match_oracle_exactly(svlib, kmax, seed):
    n = 9
    gates = random_circuit(n, 120, seed=seed, max_controls=2, max_unitary_k=3)
    ref = [a for (a, _, _, _) in oracle.fuse(n, gates, kmax)] + [len(gates)]
    for dt in (B.SV_C64, B.SV_C128):
        nb, ns, starts = B.sv_plan_info(n, dt, gates, fuse_max_k=kmax)
        assert starts == ref
        assert nb == len(ref) - 1


def test_fusion_blocks_on_the_workloads(svlib):
    for n, gates in [(12, layered_ry_rz_cnot(12, 10, 0)), (22, fused_layered_u3_cz(22, 20, 0)),
                     (20, hea_ring(20, 10)), (10, precision_sweep(10, 40, 20, 0))]:
        params = np.zeros(800)
        for k in (2, 5):
            ref = [a for (a, _, _, _) in oracle.fuse(n, gates, k, params)] + [len(gates)]
            assert B.sv_plan_info(n, B.SV_C64, gates, params, fuse_max_k=k)[2] == ref


def test_one_op_per_pass_makes_one_pass_per_gate(svlib):
    gates = fused_layered_u3_cz(16, 2, 0)
    nb, ns, _ = B.sv_plan_info(16, B.SV_C64, gates, ops_per_pass=1)
    assert ns == len(gates) == nb
    nb, ns, _ = B.sv_plan_info(16, B.SV_C64, gates)
    assert ns < len(gates) // 4


@pytest.mark.parametrize("n,depth", [(16, 20), (20, 30), (24, 40)])
def test_pass_counts_of_layered_circuits(svlib, n, depth):
    """Pass counts of the scheduler on the two layered families (host only):
    U3 + CNOT-ladder serving circuits and the 30-qubit U3 + CZ circuit.  The
    one-qubit split must not fragment the greedy passes; the serving counts
    are the whole-gate schedule's (or fewer)."""
    from workloads import serving_circuit
    whole = {(16, 20): 8, (20, 30): 57, (24, 40): 91}[(n, depth)]
    # (serving states of 21 to 25 qubits run 13-qubit tiles: the TMA pass is
    # off while a serving session is live)
    _, ns, _ = B.sv_plan_info(n, B.SV_C64, serving_circuit(n, depth, 3), fuse_max_k=5, tile_qubits=13)
    assert ns <= whole
    if n == 24:  # 30 qubits run 12-qubit tiles (states of 26 qubits and more)
        _, ns30, _ = B.sv_plan_info(30, B.SV_C64, fused_layered_u3_cz(30, 20, 0), fuse_max_k=5)
        assert ns30 <= 38


def _err(fn):
    with pytest.raises(B.SvError) as e:
        fn()
    return e.value.name


def test_boundary_rejects_bad_gates(svlib):
    plan = lambda g, **kw: B.sv_plan_info(4, B.SV_C64, g, **kw)
    assert _err(lambda: plan([Gate("h", [4])])) == "SV_ERR_INVALID"
    assert _err(lambda: plan([Gate("x", [1], [1])])) == "SV_ERR_INVALID"
    assert _err(lambda: plan([Gate("swap", [0, 0])])) == "SV_ERR_INVALID"
    assert _err(lambda: plan([Gate("rx", [0], params=[0.0], slots=[3])], param_values=[0.1])) == \
        "SV_ERR_UNBOUND_PARAM"
    assert _err(lambda: plan([Gate("rx", [0], params=[0.0], slots=[0])])) == "SV_ERR_UNBOUND_PARAM"
    assert _err(lambda: plan([Gate("unitary", [0], matrix=np.array([[1, 1], [0, 1]]))])) == "SV_ERR_INVALID"
    assert _err(lambda: plan([Gate("h", [0])], fuse_max_k=1)) == "SV_ERR_INVALID"
    assert _err(lambda: plan([Gate("h", [0])], fuse_max_k=6)) == "SV_ERR_INVALID"
    assert _err(lambda: B.sv_plan_info(0, B.SV_C64, [])) == "SV_ERR_INVALID"
    assert _err(lambda: B.sv_plan_info(35, B.SV_C64, [])) == "SV_ERR_INVALID"
    assert _err(lambda: B.sv_plan_info(4, 7, [])) == "SV_ERR_INVALID"
    # a valid plan after the failures still works, and the error text names the gate
    assert plan([Gate("h", [0])])[0] == 1
    with pytest.raises(B.SvError) as e:
        plan([Gate("h", [0]), Gate("h", [9])])
    assert "gate 1" in str(e.value)


def test_host_pointer_is_rejected_before_any_launch(svlib):
    # a host buffer passed as the state must be refused at the boundary (it
    # would otherwise be dereferenced by a kernel); on a machine without a GPU
    # the pointer query itself fails, which is also a refusal
    buf = np.zeros(16, dtype=np.complex64)
    st = svlib.sv_init_basis(ctypes.c_void_p(buf.ctypes.data), 4, B.SV_C64, 0, None)
    assert st in (1, 4)  # SV_ERR_INVALID, or SV_ERR_CUDA when no driver is present


def test_tile_width_option(svlib):
    """sv_exec_opts.tile_qubits: 0 lets the library choose; 8..13 (complex64)
    or 8..11 (complex128) forces the width; anything else is rejected before
    any planning.  A narrower tile holds fewer qubits, so it never needs fewer
    passes on the same circuit."""
    n = 22
    g = fused_layered_u3_cz(n, 6, seed=1)
    _, auto, _ = B.sv_plan_info(n, B.SV_C64, g, fuse_max_k=5)
    _, t13, _ = B.sv_plan_info(n, B.SV_C64, g, fuse_max_k=5, tile_qubits=13)
    _, t12, _ = B.sv_plan_info(n, B.SV_C64, g, fuse_max_k=5, tile_qubits=12)
    _, t8, _ = B.sv_plan_info(n, B.SV_C64, g, fuse_max_k=5, tile_qubits=8)
    assert t8 >= t12 >= t13 >= 1
    # 22 qubits: 12-qubit tiles while the compiled pass kernels are on (the
    # TMA pass with compiled programs), 13 with them off
    jit = B.sv_jit_info()
    assert auto == (t12 if jit["mode"] != 0 and jit["available"] else t13)
    B.sv_jit_set_mode(0)
    try:
        assert B.sv_plan_info(n, B.SV_C64, g, fuse_max_k=5)[1] == t13
    finally:
        B.sv_jit_set_mode(-1)
    _, c11, _ = B.sv_plan_info(n, B.SV_C128, g, fuse_max_k=5, tile_qubits=11)
    assert c11 >= 1
    for dt, bad in ((B.SV_C64, 7), (B.SV_C64, 14), (B.SV_C128, 12), (B.SV_C64, -1)):
        with pytest.raises(B.SvError):
            B.sv_plan_info(n, dt, g, fuse_max_k=5, tile_qubits=bad)
    # capped at the state size: a 6-qubit state plans with any legal width
    _, small, _ = B.sv_plan_info(6, B.SV_C64, fused_layered_u3_cz(6, 3, seed=2), fuse_max_k=5, tile_qubits=12)
    assert small == 1


def test_double_excitation_lowering_identity():
    """The adjoint runs a double excitation EXC2(theta) on (t0, t1, t2, t3) as
    C^dag RY(theta)[t0 | t1 = 0, t2 = 1, t3 = 0] C with C = X(t0) CNOT(t0->t2)
    CNOT(t2->t3) CNOT(t0->t1) (rightmost first).  The oracle confirms the
    identity on random states, with and without an extra control."""
    n = 6
    rng = np.random.default_rng(3)
    for t, ctrl in (([0, 1, 2, 3], []), ([4, 0, 5, 2], []), ([1, 3, 5, 0], [4]), ([2, 5, 0, 4], [3])):
        th = float(rng.uniform(0, 2 * np.pi))
        for cs in ([1] * len(ctrl), [0] * len(ctrl)):
            init = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
            init /= np.linalg.norm(init)
            direct = oracle.run(n, [Gate("exc2", t, ctrl, cs, params=[th])], init=init.copy())
            t0, t1, t2, t3 = t
            perm = [Gate("x", [t1], [t0]), Gate("x", [t3], [t2]), Gate("x", [t2], [t0]), Gate("x", [t0])]
            ry = Gate("ry", [t0], [t1, t2, t3] + ctrl, [0, 1, 0] + cs, params=[th])
            lowered = oracle.run(n, perm + [ry] + perm[::-1], init=init.copy())
            assert np.abs(direct - lowered).max() < 1e-13


def test_host_state_arrays_are_checked_before_the_call(svlib):
    """sv_run_host and SvState.set copy 2^n amplitudes of the dtype, so the
    binding refuses a host array that is shorter, of another dtype, strided or
    (for state_out) read-only before anything reaches the library."""
    n = 4
    good = np.zeros(2 ** n, dtype=np.complex64)
    ro = np.zeros(2 ** n, dtype=np.complex64)
    ro.flags.writeable = False
    bad_in = [np.zeros(2 ** n - 1, dtype=np.complex64), np.zeros(2 ** n, dtype=np.complex128),
              np.zeros(2 ** (n + 1), dtype=np.complex64)[::2], [0j] * 2 ** n]
    for b in bad_in:
        with pytest.raises(B.SvError) as e:
            B.sv_run_host(n, B.SV_C64, [], state_in=b)
        assert e.value.status == 1
        with pytest.raises(B.SvError):
            B.sv_run_host(n, B.SV_C64, [], state_out=b)
    with pytest.raises(B.SvError):
        B.sv_run_host(n, B.SV_C64, [], state_out=ro)
    assert B._host_state(good, n, B.SV_C64, "x").value == good.ctypes.data
    assert B._host_state(ro, n, B.SV_C64, "x").value == ro.ctypes.data  # reading is fine
