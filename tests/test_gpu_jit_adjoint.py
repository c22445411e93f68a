"""GPU checks of the adjoint's batched passes compiled at run time.

A compiled batched kernel runs the same register and shared-memory functions
as the interpreting one, in the same order, with every op field a constant;
so values and gradients agree bit for bit with the interpreted ones (which
the oracle tests of the adjoint bound), on every generator family, with
controls, shared slots, checkpoints and tiles too small for register phases.
"""

import math

import numpy as np
import pytest

import oracle
from paper_2608_09733_gb300 import binding as B
from workloads import Gate, hea_hamiltonian, hea_params, hea_ring, random_pauli_terms

pytestmark = pytest.mark.gpu

TOL = {B.SV_C64: 1e-4, B.SV_C128: 1e-10}


def grads(mode, n, dt, gates, th, terms, ckpt):
    B.sv_jit_set_mode(mode)
    try:
        before = B.sv_jit_info()["launches"]
        val, grad = B.sv_adjoint_grad(n, dt, gates, th, terms, checkpoint_every=ckpt)
        launches = B.sv_jit_info()["launches"] - before
    finally:
        B.sv_jit_set_mode(-1)
    return val, grad, launches


def mixed_circuit(n, seed):
    rng = np.random.default_rng(seed)
    gates = [Gate("h", [q]) for q in range(n)]
    fams = ["rx", "ry", "rz", "p", "rxx", "ryy", "rzz"]
    for i in range(48):
        f = fams[i % len(fams)]
        k = 2 if f in ("rxx", "ryy", "rzz") else 1
        qs = [int(v) for v in rng.permutation(n)[:k + 1]]
        ctrl = qs[k:] if i % 3 == 0 else []
        gates.append(Gate(f, qs[:k], ctrl, [int(rng.integers(0, 2))] * len(ctrl), params=[0.0],
                          slots=[int(rng.integers(0, 9))]))
        if i % 5 == 0:
            gates.append(Gate("x", [qs[0]], [qs[-1]] if qs[-1] != qs[0] else []))
        if i % 7 == 0:
            gates.append(Gate("swap", [qs[0], (qs[0] + 1) % n]))
        if i % 11 == 0:
            gates.append(Gate("u3", [qs[0]], params=[0.3, 1.1, -0.4]))
    return gates


@pytest.mark.parametrize("dt", [B.SV_C64, B.SV_C128])
@pytest.mark.parametrize("n,ckpt", [(14, 0), (14, 56), (3, 7)])
def test_hea_compiled_equals_interpreted(svlib, cuda_dev, dt, n, ckpt):
    layers, batch = 3, 4
    gates = hea_ring(n, layers)
    terms = hea_hamiltonian(n, 0.7)
    P = 2 * n * layers
    th = hea_params(batch, P, seed=21)
    v0, g0, l0 = grads(0, n, dt, gates, th, terms, ckpt)
    v1, g1, l1 = grads(2, n, dt, gates, th, terms, ckpt)
    assert l0 == 0 and l1 > 0
    assert np.array_equal(v0, v1) and np.array_equal(g0, g1)
    v_ref, g_ref = oracle.adjoint_grad(n, gates, th[0], terms, P)
    assert abs(v1[0] - v_ref) < TOL[dt] and np.max(np.abs(g1[0] - g_ref)) < TOL[dt]


@pytest.mark.parametrize("dt", [B.SV_C64, B.SV_C128])
def test_every_family_compiled_equals_interpreted(svlib, cuda_dev, dt):
    n = 9
    gates = mixed_circuit(n, 8)
    terms = random_pauli_terms(n, 9, seed=6)
    th = np.random.default_rng(2).random((3, 9)) * 2 * math.pi
    v0, g0, _ = grads(0, n, dt, gates, th, terms, 13)
    v1, g1, l1 = grads(2, n, dt, gates, th, terms, 13)
    assert l1 > 0
    assert np.array_equal(v0, v1) and np.array_equal(g0, g1)
    for b in range(3):
        v_ref, g_ref = oracle.adjoint_grad(n, gates, th[b], terms, 9)
        assert abs(v1[b] - v_ref) < TOL[dt] and np.max(np.abs(g1[b] - g_ref)) < TOL[dt]


def test_excitations_compiled_equals_interpreted(svlib, cuda_dev):
    n = 8
    gates = [Gate("x", [0]), Gate("x", [1]), Gate("x", [4])]
    gates += [Gate("exc1", [0, 2], params=[0.0], slots=[0]), Gate("exc2", [0, 1, 2, 3], params=[0.0], slots=[1]),
              Gate("exc1", [4, 5], params=[0.0], slots=[2]), Gate("exc2", [4, 6, 5, 7], params=[0.0], slots=[3]),
              Gate("ry", [3], params=[0.0], slots=[0])]
    terms = random_pauli_terms(n, 7, seed=3)
    th = np.random.default_rng(4).random((2, 4)) * 2 * math.pi
    v0, g0, _ = grads(0, n, B.SV_C64, gates, th, terms, 0)
    v1, g1, l1 = grads(2, n, B.SV_C64, gates, th, terms, 0)
    assert l1 > 0
    assert np.array_equal(v0, v1) and np.array_equal(g0, g1)


def test_second_call_compiles_by_default(svlib, cuda_dev):
    n, layers, batch = 12, 2, 3
    gates = hea_ring(n, layers)
    terms = hea_hamiltonian(n, 0.7)
    th = hea_params(batch, 2 * n * layers, seed=5)
    v0, g0, l0 = grads(1, n, B.SV_C64, gates, th, terms, 0)
    th2 = hea_params(batch, 2 * n * layers, seed=6)  # other angles, same template
    v1, g1, l1 = grads(1, n, B.SV_C64, gates, th2, terms, 0)
    v2, g2, l2 = grads(0, n, B.SV_C64, gates, th2, terms, 0)
    assert l0 == 0 and l1 > 0 and l2 == 0
    assert np.array_equal(v1, v2) and np.array_equal(g1, g2)
