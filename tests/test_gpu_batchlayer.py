"""BatchLayer (Sec. 5.4): a fixed template whose first parameter slots take
data and the rest trainable weights, evaluated as one batched state with
per-qubit <Z> readout; backward is one batched adjoint pass with the
Hamiltonian sum_q (dL/d<Z_q>_b) Z_q for row b.  Checked against the oracle
row by row, and by finite differences through torch."""
import numpy as np
import pytest

import oracle
import paper_2608_09733_gb300 as sv
from paper_2608_09733_gb300.binding import SvError
from workloads import Gate, Term

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def template(n, layers):
    """Angle encoding RY(x_q) (slots 0..n-1), then per layer RY, RZ weights
    on every qubit and a CNOT ring."""
    gates, slot = [], n
    for q in range(n):
        gates.append(Gate("ry", [q], slots=[q]))
    for _ in range(layers):
        for q in range(n):
            gates.append(Gate("ry", [q], slots=[slot]))
            gates.append(Gate("rz", [q], slots=[slot + 1]))
            slot += 2
        for q in range(n):
            gates.append(Gate("x", [(q + 1) % n], controls=[q]))
    return gates, slot


def _rows(n, n_par, batch, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, 2 * np.pi, size=(batch, n_par))


@pytest.mark.parametrize("dtype,tol", [(sv.SV_C64, 2e-5), (sv.SV_C128, 1e-12)])
def test_batch_expect_z_matches_oracle(svlib, cuda_dev, dtype, tol):
    n, batch = 10, 6
    gates, P = template(n, 3)
    params = _rows(n, P, batch, 1)
    z = sv.sv_batch_expect_z(n, dtype, gates, params)
    for b in range(batch):
        per, s = oracle.expect_z_all(oracle.run(n, gates, params[b]), n)
        assert np.abs(z[b, :n] - per).max() < tol
        assert abs(z[b, n] - s) < tol


@pytest.mark.parametrize("dtype,tol", [(sv.SV_C64, 1e-4), (sv.SV_C128, 1e-10)])
def test_row_hamiltonian_gradients_match_oracle(svlib, cuda_dev, dtype, tol):
    n, batch = 9, 5
    gates, P = template(n, 2)
    params = _rows(n, P, batch, 2)
    v = np.random.default_rng(3).normal(size=(batch, n))
    zterms = [Term("Z", [q], 1.0) for q in range(n)]
    val, grad = sv.sv_adjoint_grad_rows(n, dtype, gates, params, zterms, v)
    for b in range(batch):
        rv, rg = oracle.adjoint_grad(n, gates, params[b], [Term("Z", [q], v[b, q]) for q in range(n)], P)
        assert abs(val[b] - rv) < tol
        assert np.abs(grad[b] - rg).max() < tol


def test_row_coefficients_with_x_terms(svlib, cuda_dev):
    # mixed terms, every X-mask inside one tile
    n, batch = 8, 4
    gates, P = template(n, 2)
    params = _rows(n, P, batch, 4)
    terms = [Term("ZZ", [0, 1], 1.0), Term("X", [3], 1.0), Term("XY", [2, 7], 1.0), Term("Y", [5], 1.0)]
    c = np.random.default_rng(5).normal(size=(batch, len(terms)))
    val, grad = sv.sv_adjoint_grad_rows(n, sv.SV_C128, gates, params, terms, c)
    for b in range(batch):
        tb = [Term(t.paulis, t.qubits, c[b, j]) for j, t in enumerate(terms)]
        rv, rg = oracle.adjoint_grad(n, gates, params[b], tb, P)
        assert abs(val[b] - rv) < 1e-10 and np.abs(grad[b] - rg).max() < 1e-10


def test_row_coefficients_reject_wide_x_masks(svlib, cuda_dev):
    n = 20
    gates = [Gate("ry", [q], slots=[q]) for q in range(n)]
    wide = [Term("X" * 10, list(range(5, 15)), 1.0)]
    with pytest.raises(SvError):
        sv.sv_adjoint_grad_rows(n, sv.SV_C64, gates, _rows(n, n, 2, 6), wide, np.ones((2, 1)))


def test_layer_gradcheck_c128(svlib, cuda_dev):
    n, layers, batch = 5, 2, 3
    gates, P = template(n, layers)
    layer = sv.BatchLayer(gates, n, n_data=n, n_weights=P - n, dtype=sv.SV_C128, seed=1)
    x = torch.tensor(_rows(n, n, batch, 7), dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda xx, ww: sv.autograd._BatchLayerFn.apply(xx, ww, n, sv.SV_C128,
                                                                                    layer.gates, 0),
                                    (x, layer.weight), eps=1e-6, atol=1e-6)


def test_layer_forward_backward_matches_oracle(svlib, cuda_dev):
    n, layers, batch = 7, 2, 4
    gates, P = template(n, layers)
    layer = sv.BatchLayer(gates, n, n_data=n, n_weights=P - n, dtype=sv.SV_C64, seed=2)
    x = torch.tensor(_rows(n, n, batch, 8), dtype=torch.float64, requires_grad=True)
    target = torch.tensor(np.random.default_rng(9).normal(size=(batch, n)))
    out = layer(x)
    loss = (out * target).sum()
    loss.backward()
    w = layer.weight.detach().numpy()
    gx, gw = np.zeros((batch, n)), np.zeros(P - n)
    for b in range(batch):
        pb = np.concatenate([x.detach().numpy()[b], w])
        per, _ = oracle.expect_z_all(oracle.run(n, gates, pb), n)
        assert np.abs(out.detach().numpy()[b] - per).max() < 2e-5
        _, g = oracle.adjoint_grad(n, gates, pb, [Term("Z", [q], float(target[b, q])) for q in range(n)], P)
        gx[b], gw = g[:n], gw + g[n:]
    assert np.abs(x.grad.numpy() - gx).max() < 1e-4
    assert np.abs(layer.weight.grad.numpy() - gw).max() < 1e-4


def test_classifier_trains(svlib, cuda_dev):
    # angle encoding -> entangler -> per-qubit <Z> -> linear head, on a toy
    # two-class problem: a few Adam steps lower the loss
    torch.manual_seed(0)
    n, layers, batch = 4, 2, 32
    gates, P = template(n, layers)
    model = torch.nn.Sequential(torch.nn.Linear(2, n, dtype=torch.float64),
                                sv.BatchLayer(gates, n, n_data=n, n_weights=P - n, dtype=sv.SV_C64, seed=3),
                                torch.nn.Linear(n, 2, dtype=torch.float64))
    rng = np.random.default_rng(10)
    X = torch.tensor(rng.normal(size=(batch, 2)))
    y = torch.tensor((X[:, 0] * X[:, 1] > 0).numpy().astype(np.int64))
    opt = torch.optim.Adam(model.parameters(), lr=0.05)
    losses = []
    for _ in range(25):
        opt.zero_grad()
        loss = torch.nn.functional.cross_entropy(model(X), y)
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert losses[-1] < losses[0] - 0.05
