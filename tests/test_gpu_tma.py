"""GPU parity of the TMA pass kernel (complex64 states with 12-qubit tiles and
at least 2^9 of them) against the oracle, element by element.

The library picks that kernel for complex64 states of 26 qubits and more;
here the tile width option forces 12-qubit tiles on 21- to 24-qubit states
so that the oracle can check every amplitude.  A CTA refills its ring of
stages only when it has more tiles than stages, so the 24- and 26-qubit
cases (27 and 108 tiles per CTA on 152 SMs) are the ones that exercise the
refill path; the 21- and 22-qubit ones fit the first fill.  Every op kind the pass
programs have (rotations and phase tables, bit flips and swaps, dense and
diagonal ops with controls inside and outside the tile, fused dense blocks
in shared memory) is covered, and the kernel is checked to give the same
bits as the cp.async pass kernel on the same programs.
"""

import os

import numpy as np
import pytest

import oracle
from paper_2608_09733_gb300 import binding as B
from workloads import fused_layered_u3_cz, random_circuit, serving_circuit

pytestmark = pytest.mark.gpu

TOL_C64 = 1e-5


def run(n, gates, fuse=0, block_mode=0, tile=12, tma=True):
    import torch
    old = os.environ.get("SV_SWEEP_TMA")
    os.environ["SV_SWEEP_TMA"] = "1" if tma else "0"
    try:
        st = torch.empty(2 ** n, dtype=torch.complex64, device="cuda")
        B.sv_init_basis(st, 0)
        B.sv_apply_circuit_ex(st, gates, fuse_max_k=fuse, block_mode=block_mode, tile_qubits=tile)
        torch.cuda.synchronize()
    finally:
        if old is None:
            del os.environ["SV_SWEEP_TMA"]
        else:
            os.environ["SV_SWEEP_TMA"] = old
    return st.cpu().numpy()


def maxabs(a, ref):
    return float(np.max(np.abs(a.astype(np.complex128) - ref)))


@pytest.mark.parametrize("n,ng", [(21, 160), (22, 160), (24, 100)])
def test_tma_pass_random_circuits_all_families(svlib, cuda_dev, n, ng):
    gates = random_circuit(n, ng, seed=700 + n, max_controls=3, max_unitary_k=5)
    ref = oracle.run(n, gates)
    for fuse, mode in ((0, 0), (5, 0), (5, 1)):
        _, passes, _ = B.sv_plan_info(n, B.SV_C64, gates, fuse_max_k=fuse, block_mode=mode, tile_qubits=12)
        assert passes >= 2
        got = run(n, gates, fuse=fuse, block_mode=mode)
        assert maxabs(got, ref) < TOL_C64, (fuse, mode, maxabs(got, ref))


def test_tma_pass_layered_u3_cz_22q(svlib, cuda_dev):
    n = 22
    gates = fused_layered_u3_cz(n, 20, seed=3)
    ref = oracle.run(n, gates)
    got = run(n, gates, fuse=5)
    assert maxabs(got, ref) < TOL_C64, maxabs(got, ref)


def test_tma_pass_serving_circuit_21q(svlib, cuda_dev):
    n = 21
    gates = serving_circuit(n, 12, seed=5)
    ref = oracle.run(n, gates)
    got = run(n, gates, fuse=5)
    assert maxabs(got, ref) < TOL_C64, maxabs(got, ref)


@pytest.mark.parametrize("n,fuse", [(22, 0), (22, 5), (26, 0), (26, 5)])
def test_tma_pass_bitwise_equals_cp_async_pass(svlib, cuda_dev, n, fuse):
    """The two kernels interpret the same programs with the same arithmetic;
    only the tile movement differs, so the states agree bit for bit."""
    gates = random_circuit(n, 120, seed=31 + fuse, max_controls=2, max_unitary_k=3)
    a = run(n, gates, fuse=fuse, tma=True)
    b = run(n, gates, fuse=fuse, tma=False)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_tma_pass_layered_bitwise_equals_cp_async_pass_26q(svlib, cuda_dev):
    n = 26
    gates = fused_layered_u3_cz(n, 8, seed=4)
    a = run(n, gates, fuse=5, tma=True)
    b = run(n, gates, fuse=5, tma=False)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_tma_pass_deterministic(svlib, cuda_dev):
    n = 24
    gates = fused_layered_u3_cz(n, 6, seed=9)
    a = run(n, gates, fuse=5)
    b = run(n, gates, fuse=5)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
