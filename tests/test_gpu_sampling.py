"""Measurement on the GPU (sv_probabilities, sv_sample) against the oracle on
the same state: the draws are exact integer inverse-CDF lookups, so the
indices must match bit for bit; probabilities match to the last bit before
normalisation."""
import numpy as np
import pytest

import oracle
import paper_2608_09733_gb300 as sv
from paper_2608_09733_gb300.binding import SvError
from workloads import Gate, fused_layered_u3_cz, random_circuit

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _state(n, dtype, circ):
    tdt = torch.complex64 if dtype == sv.SV_C64 else torch.complex128
    st = torch.empty(2 ** n, dtype=tdt, device="cuda")
    sv.sv_init_basis(st, 0)
    sv.sv_apply_circuit(st, circ, fuse_max_k=5)
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("dtype", [sv.SV_C64, sv.SV_C128])
@pytest.mark.parametrize("n,shots", [(5, 4000), (9, 20000), (14, 100000), (22, 100000)])
def test_sample_matches_oracle_exactly(svlib, cuda_dev, dtype, n, shots):
    st = _state(n, dtype, random_circuit(n, 150, seed=n, max_controls=1, max_unitary_k=2))
    host = st.cpu().numpy().astype(np.complex128)
    u = np.random.default_rng(100 + n).random(shots)
    u[:3] = [0.0, 0.5, 1.0 - 2.0 ** -53]
    got = sv.sv_sample(st, u)
    ref = oracle.sample(host, n, u)
    assert (got == ref).all()


@pytest.mark.parametrize("dtype", [sv.SV_C64, sv.SV_C128])
def test_probabilities_match_oracle(svlib, cuda_dev, dtype):
    n = 16
    st = _state(n, dtype, random_circuit(n, 200, seed=3))
    host = st.cpu().numpy().astype(np.complex128)
    raw = sv.sv_probabilities(st, normalise=False).cpu().numpy()
    assert (raw == oracle.probabilities(host, n, normalise=False)).all()
    nrm = sv.sv_probabilities(st).cpu().numpy()
    assert np.allclose(nrm, oracle.probabilities(host, n), rtol=1e-13, atol=1e-300)
    assert abs(nrm.sum() - 1.0) < 1e-12


def test_sample_into_device_memory_and_edges(svlib, cuda_dev):
    n = 12
    st = _state(n, sv.SV_C64, random_circuit(n, 60, seed=5))
    u = np.random.default_rng(7).random(3000)
    dev = torch.empty(u.size, dtype=torch.int64, device="cuda")
    sv.sv_sample(st, u, out=dev)
    torch.cuda.synchronize()
    assert (dev.cpu().numpy().astype(np.uint64) == sv.sv_sample(st, u)).all()
    assert sv.sv_sample(st, np.zeros(0)).size == 0
    with pytest.raises(SvError):
        sv.sv_sample(st, np.array([0.2, 1.0]))
    with pytest.raises(SvError):
        sv.sv_sample(st, np.array([-0.1]))
    zero = torch.zeros(2 ** n, dtype=torch.complex64, device="cuda")
    with pytest.raises(SvError):
        sv.sv_sample(zero, np.array([0.3]))
    small = torch.zeros(2 ** 4, dtype=torch.complex64, device="cuda")
    with pytest.raises(SvError):
        sv.sv_sample(small, np.array([0.3]))


def test_basis_state_at_26_qubits(svlib, cuda_dev):
    n, k = 26, 0x2A5F3C1
    st = torch.zeros(2 ** n, dtype=torch.complex64, device="cuda")
    sv.sv_init_basis(st, k)
    u = np.random.default_rng(1).random(50000)
    assert (sv.sv_sample(st, u) == k).all()


def test_product_state_marginals_at_30_qubits(svlib, cuda_dev):
    # RY(theta_q) on every qubit of |0..0>: bit q is 1 with probability
    # sin^2(theta_q / 2), independently (a property that holds at any size)
    n, shots = 30, 1 << 20
    theta = np.linspace(0.2, 2.9, n)
    st = _state(n, sv.SV_C64, [Gate("ry", [q], params=[float(theta[q])]) for q in range(n)])
    idx = sv.sv_sample(st, np.random.default_rng(2).random(shots))
    bits = ((idx[:, None] >> np.arange(n, dtype=np.uint64)) & np.uint64(1)).astype(np.float64).mean(axis=0)
    expect = np.sin(theta / 2) ** 2
    assert np.abs(bits - expect).max() < 6 * 0.5 / np.sqrt(shots)
    del st
    torch.cuda.empty_cache()
