"""Checkpoint policies of the adjoint (Sec. 7.3: none, a user interval, or
automatic placement; discarded states recomputed in backward): every policy
gives the oracle's gradients."""
import numpy as np
import pytest

import oracle
import paper_2608_09733_gb300 as sv
from workloads import hea_hamiltonian, hea_params, hea_ring

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

POLICIES = [
    dict(checkpoint_every=0),
    dict(checkpoint_every=12),                                # keep every segment start
    dict(checkpoint_every=12, stored_states=0),               # recompute each from |0..0>
    dict(checkpoint_every=12, stored_states=1),
    dict(checkpoint_every=7, stored_states=3),
    dict(checkpoint_every=12, memory_budget_bytes=2.5 * 8 * 2 ** 12 * 3),  # automatic: two states fit
]


@pytest.mark.parametrize("dtype,tol", [(sv.SV_C64, 1e-4), (sv.SV_C128, 1e-10)])
@pytest.mark.parametrize("policy", POLICIES, ids=[str(p) for p in POLICIES])
def test_policies_match_oracle(svlib, cuda_dev, dtype, tol, policy):
    n, layers, batch = 12, 4, 3
    gates, H = hea_ring(n, layers), hea_hamiltonian(n)
    P = 2 * n * layers
    params = hea_params(batch, P, seed=5)
    val, grad = sv.sv_adjoint_grad_ex(n, dtype, gates, params, H, **policy)
    for b in range(batch):
        rv, rg = oracle.adjoint_grad(n, gates, params[b], H, P)
        assert abs(val[b] - rv) < tol
        assert np.abs(grad[b] - rg).max() < tol


def test_recompute_equals_stored_at_20_qubits(svlib, cuda_dev):
    n, layers, batch = 20, 6, 4
    gates, H = hea_ring(n, layers), hea_hamiltonian(n)
    params = hea_params(batch, 2 * n * layers, seed=6)
    _, g_all = sv.sv_adjoint_grad_ex(n, sv.SV_C64, gates, params, H, checkpoint_every=40)
    _, g_re = sv.sv_adjoint_grad_ex(n, sv.SV_C64, gates, params, H, checkpoint_every=40, stored_states=1)
    assert np.abs(g_all - g_re).max() < 1e-4
