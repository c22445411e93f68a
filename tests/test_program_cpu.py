"""The pass kernel's programs, run on the host (sv_emulate_apply), against the
oracle: checks the program builder (tiles, register phases, rotation split,
phase tables with selector variants, diagonal placement, dispatch words)
without a GPU.  complex128 programs carry double coefficients; complex64
programs carry float coefficients, so their tolerance is the float rounding
of the coefficients."""
import numpy as np
import pytest

import oracle
import paper_2608_09733_gb300 as sv
from workloads import (fused_layered_u3_cz, ghz_circuit, hea_params, hea_ring, layered_ry_rz_cnot,
                       precision_sweep, qft_circuit, random_circuit)

TOL = {sv.SV_C128: 1e-12, sv.SV_C64: 2e-6}


def _emulate(n, circ, dtype, params=None, **kw):
    st = np.zeros(2 ** n, dtype=np.complex128)
    st[0] = 1.0
    return sv.sv_emulate_apply(st, n, dtype, circ, param_values=params, **kw)


CASES = [
    ("layered_u3_cz", 16, lambda: fused_layered_u3_cz(16, 8, 3)),
    ("layered_u3_cz_small", 7, lambda: fused_layered_u3_cz(7, 10, 4)),
    ("ry_rz_cnot", 14, lambda: layered_ry_rz_cnot(14, 6, 5)),
    ("random_controls", 15, lambda: random_circuit(15, 250, seed=6, max_controls=2, max_unitary_k=3)),
    ("random_small", 6, lambda: random_circuit(6, 200, seed=7, max_controls=3, max_unitary_k=4)),
    ("ghz", 17, lambda: ghz_circuit(17)),
    ("qft", 12, lambda: qft_circuit(12, with_swaps=True)),
    ("precision_sweep", 16, lambda: precision_sweep(16, 200, 8)),
]


@pytest.mark.parametrize("dtype", [sv.SV_C64, sv.SV_C128])
@pytest.mark.parametrize("name,n,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("fuse", [0, 5])
def test_programs_match_oracle(name, n, make, dtype, fuse):
    circ = make()
    got = _emulate(n, circ, dtype, fuse_max_k=fuse)
    ref = oracle.run(n, circ)
    assert np.abs(got - ref).max() <= TOL[dtype]


def _closing_phase_circuit(n, layers, seed):
    """Layers of one-qubit gates of every shape the rotation split meets --
    general U3, diagonal (theta = 0), anti-diagonal (theta = pi), real, phase
    and Clifford gates -- with CZ, CP and controlled RZ between near and far
    qubits, so that closing phases and other diagonals must wait for later
    passes (17 qubits: several 12-qubit tiles)."""
    from workloads.circuits import Gate
    rng = np.random.default_rng(seed)
    one = ["u3", "u3", "u3z", "u3x", "h", "s", "t", "sx", "rx", "ry", "rz", "p", "y"]
    gates = []
    for _ in range(layers):
        for q in range(n):
            kind = one[rng.integers(len(one))]
            if kind == "u3z":
                gates.append(Gate("u3", [q], params=[0.0, *rng.uniform(-3, 3, 2)]))
            elif kind == "u3x":
                gates.append(Gate("u3", [q], params=[np.pi, *rng.uniform(-3, 3, 2)]))
            elif kind == "u3":
                gates.append(Gate("u3", [q], params=list(rng.uniform(-3, 3, 3))))
            elif kind in ("rx", "ry", "rz", "p"):
                gates.append(Gate(kind, [q], params=[float(rng.uniform(-3, 3))]))
            else:
                gates.append(Gate(kind, [q]))
        for q in range(0, n - 1, 2):
            gates.append(Gate("z", [q + 1], controls=[q]))
        for _ in range(4):
            a, b = (int(x) for x in rng.choice(n, 2, replace=False))
            if rng.integers(2):
                gates.append(Gate("p", [a], controls=[b], params=[float(rng.uniform(-3, 3))]))
            else:
                gates.append(Gate("rz", [a], controls=[b], params=[float(rng.uniform(-3, 3))]))
    return gates


@pytest.mark.parametrize("dtype", [sv.SV_C64, sv.SV_C128])
@pytest.mark.parametrize("fuse", [0, 5])
def test_programs_closing_phases_across_passes(dtype, fuse):
    n = 17
    circ = _closing_phase_circuit(n, 6, seed=21)
    _, passes, _ = sv.sv_plan_info(n, dtype, sv.Gates(circ), fuse_max_k=fuse)
    assert passes >= 2
    got = _emulate(n, circ, dtype, fuse_max_k=fuse)
    ref = oracle.run(n, circ)
    assert np.abs(got - ref).max() <= TOL[dtype]


@pytest.mark.parametrize("dtype", [sv.SV_C64, sv.SV_C128])
def test_programs_bound_parameters(dtype):
    n = 12
    circ = hea_ring(n, 4)
    params = hea_params(1, 2 * n * 4, seed=9)[0]
    got = _emulate(n, circ, dtype, params=params)
    ref = oracle.run(n, circ, params)
    assert np.abs(got - ref).max() <= TOL[dtype]


@pytest.mark.parametrize("dtype", [sv.SV_C64, sv.SV_C128])
def test_programs_one_op_per_pass_and_dense_blocks(dtype):
    n = 15
    circ = random_circuit(n, 120, seed=11, max_controls=1, max_unitary_k=2)
    ref = oracle.run(n, circ)
    for kw in (dict(ops_per_pass=1), dict(fuse_max_k=4, block_mode=sv.SV_BLOCK_DENSE)):
        got = _emulate(n, circ, dtype, **kw)
        assert np.abs(got - ref).max() <= TOL[dtype], kw
