"""GPU parity of the batched adjoint gradient (sv_adjoint_grad) against the
oracle's adjoint, the parameter-shift rule and central finite differences.

Tolerances: complex64 values and gradients 1e-4 absolute (complex128 1e-10).
"""

import math

import numpy as np
import pytest

import oracle
from paper_2608_09733_gb300 import binding as B
from workloads import Gate, Term, hea_hamiltonian, hea_params, hea_ring, random_pauli_terms

pytestmark = pytest.mark.gpu

TOL = {B.SV_C64: 1e-4, B.SV_C128: 1e-10}


@pytest.mark.parametrize("dt", [B.SV_C64, B.SV_C128])
@pytest.mark.parametrize("ckpt", [0, 7, 36])
def test_hea_small_vs_oracle_adjoint(svlib, cuda_dev, dt, ckpt):
    n, layers, batch = 6, 3, 4
    gates = hea_ring(n, layers)
    terms = hea_hamiltonian(n, 0.7)
    P = 2 * n * layers
    th = hea_params(batch, P, seed=11)
    val, grad = B.sv_adjoint_grad(n, dt, gates, th, terms, checkpoint_every=ckpt)
    for b in range(batch):
        v_ref, g_ref = oracle.adjoint_grad(n, gates, th[b], terms, P)
        assert abs(val[b] - v_ref) < TOL[dt]
        assert np.max(np.abs(grad[b] - g_ref)) < TOL[dt]


def test_matches_parameter_shift_and_finite_differences(svlib, cuda_dev):
    n, layers = 5, 2
    gates = hea_ring(n, layers)
    terms = hea_hamiltonian(n, 0.7)
    P = 2 * n * layers
    th = hea_params(1, P, seed=3)[0]
    _, g = B.sv_adjoint_grad(n, B.SV_C128, gates, th, terms)
    g_ps = oracle.param_shift_grad(n, gates, th, terms, P)
    g_fd = oracle.fd_grad(n, gates, th, terms, P, h=1e-3)
    assert np.max(np.abs(g[0] - g_ps)) < 1e-10
    assert np.max(np.abs(g[0] - g_fd)) < 1e-5
    _, g32 = B.sv_adjoint_grad(n, B.SV_C64, gates, th, terms)
    assert np.max(np.abs(g32[0] - g_ps)) < 1e-4


@pytest.mark.parametrize("dt", [B.SV_C64, B.SV_C128])
def test_all_generator_families_controls_and_shared_slots(svlib, cuda_dev, dt):
    n = 7
    rng = np.random.default_rng(5)
    gates = [Gate("h", [q]) for q in range(n)]
    fams = ["rx", "ry", "rz", "p", "rxx", "ryy", "rzz"]
    for i in range(40):
        f = fams[i % len(fams)]
        k = 2 if f in ("rxx", "ryy", "rzz") else 1
        qs = [int(v) for v in rng.permutation(n)[:k + 1]]
        ctrl = qs[k:] if i % 3 == 0 else []
        gates.append(Gate(f, qs[:k], ctrl, [int(rng.integers(0, 2))] * len(ctrl), params=[0.0],
                          slots=[int(rng.integers(0, 9))]))
        if i % 5 == 0:
            gates.append(Gate("x", [qs[0]], [qs[-1]] if k + 1 > 1 and qs[-1] != qs[0] else []))
        if i % 7 == 0:
            gates.append(Gate("swap", [qs[0], (qs[0] + 1) % n]))
    terms = random_pauli_terms(n, 9, seed=4)
    th = rng.random((3, 9)) * 2 * math.pi
    val, grad = B.sv_adjoint_grad(n, dt, gates, th, terms, checkpoint_every=11)
    for b in range(3):
        v_ref, g_ref = oracle.adjoint_grad(n, gates, th[b], terms, 9)
        assert abs(val[b] - v_ref) < TOL[dt]
        assert np.max(np.abs(grad[b] - g_ref)) < TOL[dt]


def test_batch_rows_are_independent(svlib, cuda_dev):
    n, layers = 10, 4
    gates = hea_ring(n, layers)
    terms = hea_hamiltonian(n, 0.7)
    P = 2 * n * layers
    th = hea_params(6, P, seed=2)
    val, grad = B.sv_adjoint_grad(n, B.SV_C64, gates, th, terms, checkpoint_every=2 * 3 * n)
    v1, g1 = B.sv_adjoint_grad(n, B.SV_C64, gates, th[3:4], terms, checkpoint_every=2 * 3 * n)
    assert np.array_equal(val[3:4], v1) and np.array_equal(grad[3:4], g1)


def test_config4_reduced_12q_c64_checkpoints(svlib, cuda_dev):
    n, layers, batch = 12, 10, 8
    gates = hea_ring(n, layers)
    terms = hea_hamiltonian(n, 0.7)
    P = 2 * n * layers
    th = hea_params(batch, P, seed=0)
    val, grad = B.sv_adjoint_grad(n, B.SV_C64, gates, th, terms, checkpoint_every=2 * 3 * n)
    for b in (0, batch - 1):
        v_ref, g_ref = oracle.adjoint_grad(n, gates, th[b], terms, P)
        assert abs(val[b] - v_ref) < 1e-4
        assert np.max(np.abs(grad[b] - g_ref)) < 1e-4


def test_unsupported_and_invalid(svlib, cuda_dev):
    terms = [Term("Z", [0], 1.0)]
    with pytest.raises(B.SvError) as e:
        B.sv_adjoint_grad(1, B.SV_C64, [Gate("u3", [0], params=[0, 0, 0], slots=[0, -1, -1])], [[0.1]], terms)
    assert e.value.name == "SV_ERR_UNSUPPORTED"
    with pytest.raises(B.SvError) as e:
        B.sv_adjoint_grad(2, B.SV_C64, [Gate("rx", [0], params=[0], slots=[2])], [[0.1, 0.2]], terms)
    assert e.value.name == "SV_ERR_UNBOUND_PARAM"
    with pytest.raises(B.SvError) as e:
        B.sv_adjoint_grad(2, B.SV_C64, [Gate("rx", [0], params=[0], slots=[0])], [[0.1]], [Term("Z", [3], 1.0)])
    assert e.value.name == "SV_ERR_INVALID"


def test_torch_autograd_wrapper(svlib, cuda_dev):
    import torch
    from paper_2608_09733_gb300 import adjoint_expectation
    n, layers = 6, 2
    gates = hea_ring(n, layers)
    terms = hea_hamiltonian(n, 0.7)
    P = 2 * n * layers
    th = torch.tensor(hea_params(3, P, seed=8), dtype=torch.float64, requires_grad=True)
    f = adjoint_expectation(th, n, gates, terms, dtype=B.SV_C128)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    (f * w).sum().backward()
    for b in range(3):
        v_ref, g_ref = oracle.adjoint_grad(n, gates, th[b].detach().numpy(), terms, P)
        assert abs(float(f[b].detach()) - v_ref) < 1e-10
        assert np.max(np.abs(th.grad[b].numpy() - w[b].item() * g_ref)) < 1e-10


@pytest.mark.slow
def test_config4_full_size_one_row(svlib, cuda_dev):
    """20 qubits, 10 layers, batch 64, complex64, checkpoints every 2 layers:
    two rows against the complex128 oracle adjoint."""
    n, layers, batch = 20, 10, 64
    gates = hea_ring(n, layers)
    terms = hea_hamiltonian(n, 0.7)
    P = 2 * n * layers
    th = hea_params(batch, P, seed=0)
    val, grad = B.sv_adjoint_grad(n, B.SV_C64, gates, th, terms, checkpoint_every=2 * 3 * n)
    for b in (0, 37):
        v_ref, g_ref = oracle.adjoint_grad(n, gates, th[b], terms, P)
        assert abs(val[b] - v_ref) < 1e-4
        assert np.max(np.abs(grad[b] - g_ref)) < 1e-4
