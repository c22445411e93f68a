"""The device-array adjoint entry points (sv_adjoint_grad_device,
sv_batch_expect_z_device) and the autograd wrappers built on them: gate tables
built on the device from device parameters, per-state Hamiltonians, values
only, and the BatchLayer step with every tensor on the GPU.  Checked against
the oracle and against the host-array entry points (Sec. 4.2 gradients,
Sec. 5.4 BatchLayer)."""
import numpy as np
import pytest

import oracle
import paper_2608_09733_gb300 as sv
from workloads import Gate, Term, random_pauli_terms

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {sv.SV_C64: 1e-4, sv.SV_C128: 1e-10}


def _template(n, rng):
    """Every family the device table builder makes, with controls (some on
    |0>) and a slot shared by several gates."""
    gates = [Gate("h", [q]) for q in range(n)]
    fams = ["rx", "ry", "rz", "p", "rxx", "ryy", "rzz", "exc1", "exc2"]
    nslot = 11
    for i in range(36):
        f = fams[i % len(fams)]
        k = 4 if f == "exc2" else 2 if f in ("rxx", "ryy", "rzz", "exc1") else 1
        qs = [int(v) for v in rng.permutation(n)[:k + 1]]
        ctrl = qs[k:] if i % 4 == 0 else []
        gates.append(Gate(f, qs[:k], ctrl, [int(rng.integers(0, 2))] * len(ctrl), slots=[int(rng.integers(0, nslot))]))
        if i % 5 == 0:
            gates.append(Gate("x", [qs[0]], [qs[1]]))
    return gates, nslot


@pytest.mark.parametrize("dt", [sv.SV_C64, sv.SV_C128])
def test_device_adjoint_matches_oracle_and_host_entry_point(svlib, cuda_dev, dt):
    n, batch = 8, 4
    rng = np.random.default_rng(21)
    gates, P = _template(n, rng)
    terms = random_pauli_terms(n, 7, seed=22)
    th = rng.uniform(0, 2 * np.pi, size=(batch, P))
    pd = torch.tensor(th, dtype=torch.float64, device="cuda")
    for ck in (0, 9):
        val, grad = sv.sv_adjoint_grad_device(n, dt, gates, pd, terms, checkpoint_every=ck)
        torch.cuda.synchronize()
        v_host, g_host = sv.sv_adjoint_grad(n, dt, gates, th, terms, checkpoint_every=ck)
        assert np.abs(val.cpu().numpy() - v_host).max() < (1e-6 if dt == sv.SV_C64 else 1e-12)
        assert np.abs(grad.cpu().numpy() - g_host).max() < (1e-6 if dt == sv.SV_C64 else 1e-12)
        for b in range(batch):
            rv, rg = oracle.adjoint_grad(n, gates, th[b], terms, P)
            assert abs(float(val[b]) - rv) < TOL[dt]
            assert np.abs(grad[b].cpu().numpy() - rg).max() < TOL[dt]


@pytest.mark.parametrize("dt", [sv.SV_C64, sv.SV_C128])
def test_device_adjoint_values_only_and_row_coefficients(svlib, cuda_dev, dt):
    n, batch = 9, 3
    rng = np.random.default_rng(23)
    gates, P = _template(n, rng)
    zterms = [Term("Z", [q], 1.0) for q in range(n)]
    th = rng.uniform(0, 2 * np.pi, size=(batch, P))
    coeffs = rng.normal(size=(batch, n))
    pd = torch.tensor(th, device="cuda")
    cd = torch.tensor(coeffs, device="cuda")
    val, grad = sv.sv_adjoint_grad_device(n, dt, gates, pd, zterms, row_coeffs=cd)
    only, none = sv.sv_adjoint_grad_device(n, dt, gates, pd, zterms, row_coeffs=cd, values_only=True)
    torch.cuda.synchronize()
    assert none is None
    assert np.array_equal(only.cpu().numpy(), val.cpu().numpy())
    v_host, g_host = sv.sv_adjoint_grad_rows(n, dt, gates, th, zterms, coeffs)
    assert np.abs(val.cpu().numpy() - v_host).max() < TOL[dt]
    assert np.abs(grad.cpu().numpy() - g_host).max() < TOL[dt]
    z = sv.sv_batch_expect_z_device(n, dt, gates, pd)
    torch.cuda.synchronize()
    for b in range(batch):
        per, s = oracle.expect_z_all(oracle.run(n, gates, th[b]), n)
        assert np.abs(z[b, :n].cpu().numpy() - per).max() < TOL[dt] and abs(float(z[b, n]) - s) < TOL[dt]
        assert abs(float(val[b]) - float(np.dot(coeffs[b], per))) < TOL[dt]


def test_autograd_values_only_without_grad(svlib, cuda_dev):
    n = 6
    rng = np.random.default_rng(24)
    gates, P = _template(n, rng)
    terms = random_pauli_terms(n, 5, seed=25)
    p = torch.tensor(rng.uniform(0, 6.2, size=(2, P)), device="cuda", requires_grad=True)
    f = sv.adjoint_expectation(p, n, gates, terms, dtype=sv.SV_C128)
    f.sum().backward()
    with torch.no_grad():
        f2 = sv.adjoint_expectation(p, n, gates, terms, dtype=sv.SV_C128)
    assert f.is_cuda and p.grad.is_cuda
    assert torch.equal(f.detach(), f2)
    for b in range(2):
        rv, rg = oracle.adjoint_grad(n, gates, p[b].detach().cpu().numpy(), terms, P)
        assert abs(float(f[b].detach()) - rv) < 1e-10 and np.abs(p.grad[b].cpu().numpy() - rg).max() < 1e-10


def test_batchlayer_step_on_the_device_matches_oracle(svlib, cuda_dev):
    n, layers, batch = 7, 2, 4
    gates, slot = [Gate("ry", [q], slots=[q]) for q in range(n)], n
    for _ in range(layers):
        for q in range(n):
            gates += [Gate("ry", [q], slots=[slot]), Gate("rz", [q], slots=[slot + 1])]
            slot += 2
        gates += [Gate("x", [(q + 1) % n], controls=[q]) for q in range(n)]
    layer = sv.BatchLayer(gates, n, n_data=n, n_weights=slot - n, dtype=sv.SV_C64, seed=2).cuda()
    rng = np.random.default_rng(8)
    x = torch.tensor(rng.uniform(0, np.pi, size=(batch, n)), device="cuda", requires_grad=True)
    target = torch.tensor(rng.normal(size=(batch, n)), device="cuda")
    out = layer(x)
    (out * target).sum().backward()
    assert out.is_cuda and x.grad.is_cuda and layer.weight.grad.is_cuda
    w = layer.weight.detach().cpu().numpy()
    gx, gw = np.zeros((batch, n)), np.zeros(slot - n)
    for b in range(batch):
        pb = np.concatenate([x.detach().cpu().numpy()[b], w])
        per, _ = oracle.expect_z_all(oracle.run(n, gates, pb), n)
        assert np.abs(out.detach().cpu().numpy()[b] - per).max() < 2e-5
        _, g = oracle.adjoint_grad(n, gates, pb, [Term("Z", [q], float(target[b, q])) for q in range(n)], slot)
        gx[b], gw = g[:n], gw + g[n:]
    assert np.abs(x.grad.cpu().numpy() - gx).max() < 1e-4
    assert np.abs(layer.weight.grad.cpu().numpy() - gw).max() < 1e-4
