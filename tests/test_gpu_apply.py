"""GPU parity: gate application and expectations through the C ABI vs the oracle.

Tolerances (element by element against the complex128 oracle): complex128
states 1e-12 max-abs, complex64 states 1e-5 max-abs, complex64 expectations
1e-4.  Sizes span several tiles (a tile is 2^12 amplitudes for complex64 and
2^11 for complex128) with ragged qubit positions.
"""

import math

import numpy as np
import pytest

import oracle
from paper_2608_09733_gb300 import binding as B
from workloads import (Gate, Term, fused_layered_u3_cz, ghz_circuit, layered_ry_rz_cnot, precision_sweep,
                       qft_circuit, random_circuit, random_pauli_terms)

pytestmark = pytest.mark.gpu

TOL_STATE = {B.SV_C64: 1e-5, B.SV_C128: 1e-12}
TOL_EXPECT = {B.SV_C64: 1e-4, B.SV_C128: 1e-11}


def torch_dtype(dt):
    import torch
    return torch.complex64 if dt == B.SV_C64 else torch.complex128


def gpu_state(n, gates, dt, params=None, fuse=0, block_mode=0, ops_per_pass=0, init=None):
    import torch
    if init is None:
        st = torch.empty(2 ** n, dtype=torch_dtype(dt), device="cuda")
        B.sv_init_basis(st, 0)
    else:
        st = torch.as_tensor(init).to(torch_dtype(dt)).cuda().contiguous()
    B.sv_apply_circuit_ex(st, gates, params, fuse_max_k=fuse, block_mode=block_mode, ops_per_pass=ops_per_pass)
    torch.cuda.synchronize()
    return st


def maxabs(st, ref):
    return float(np.max(np.abs(st.cpu().numpy().astype(np.complex128) - ref)))


DTS = [B.SV_C64, B.SV_C128]


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 13, 15])
def test_random_circuits_all_families(svlib, cuda_dev, dt, n):
    gates = random_circuit(n, 150, seed=100 + n, max_controls=min(3, n - 1) if n > 1 else 0,
                           max_unitary_k=min(5, n))
    ref = oracle.run(n, gates)
    for fuse in (0, 2, 5):
        st = gpu_state(n, gates, dt, fuse=fuse)
        assert maxabs(st, ref) < TOL_STATE[dt], (fuse, maxabs(st, ref))


@pytest.mark.parametrize("dt", DTS)
def test_dense_fused_blocks_and_one_op_per_pass(svlib, cuda_dev, dt):
    n = 14
    gates = random_circuit(n, 120, seed=7, max_controls=1, max_unitary_k=2)
    ref = oracle.run(n, gates)
    for k in (2, 3, 4, 5):
        st = gpu_state(n, gates, dt, fuse=k, block_mode=B.SV_BLOCK_DENSE)
        assert maxabs(st, ref) < TOL_STATE[dt], k
    st = gpu_state(n, gates, dt, ops_per_pass=1)
    assert maxabs(st, ref) < TOL_STATE[dt]


@pytest.mark.parametrize("dt", DTS)
def test_high_qubit_targets_and_external_controls(svlib, cuda_dev, dt):
    # targets far above the tile's low qubits; controls outside the tile
    n = 17
    rng = np.random.default_rng(3)
    gates = [Gate("h", [q]) for q in range(n)]
    for _ in range(60):
        t, c1, c2 = [int(v) for v in rng.permutation(n)[:3]]
        gates.append(Gate("u3", [t], [c1, c2], [int(rng.integers(0, 2)), 1], params=list(rng.random(3) * 6)))
        gates.append(Gate("rzz", [c1, t], params=[float(rng.random() * 6)]))
        gates.append(Gate("x", [c2], [t], [0]))
        gates.append(Gate("swap", [t, c2], [c1]))
    ref = oracle.run(n, gates)
    st = gpu_state(n, gates, dt)
    assert maxabs(st, ref) < TOL_STATE[dt]


def test_config1_layered_12q_c128_state_and_z(svlib, cuda_dev):
    n = 12
    gates = layered_ry_rz_cnot(n, 10, seed=0)
    ref = oracle.run(n, gates)
    st = gpu_state(n, gates, B.SV_C128)
    assert maxabs(st, ref) < 1e-12
    z = B.sv_expect_z_all(st)
    per, s = oracle.expect_z_all(ref, n)
    assert abs(z[0] - per[0]) < 1e-12 and abs(z[n] - s) < 1e-11
    assert np.max(np.abs(z[:n] - per)) < 1e-12


@pytest.mark.parametrize("dt", DTS)
def test_config2_fused_layered_22q(svlib, cuda_dev, dt):
    n = 22
    gates = fused_layered_u3_cz(n, 20, seed=0)
    ref = oracle.run(n, gates)
    for fuse, mode in ((5, B.SV_BLOCK_AUTO), (0, B.SV_BLOCK_AUTO)):
        st = gpu_state(n, gates, dt, fuse=fuse, block_mode=mode)
        err = maxabs(st, ref)
        assert err < TOL_STATE[dt], (fuse, mode, err)
        ov = abs(np.vdot(ref, st.cpu().numpy().astype(np.complex128)))
        assert abs(ov - 1) < (1e-5 if dt == B.SV_C64 else 1e-12)


@pytest.mark.parametrize("dt", DTS)
def test_config3_precision_sweep_20q(svlib, cuda_dev, dt):
    n = 20
    gates = precision_sweep(n, 400, 200, seed=0)
    for depth in (100, 200, 600):
        ref = oracle.run(n, gates[:depth])
        st = gpu_state(n, gates[:depth], dt)
        err = maxabs(st, ref)
        assert err < TOL_STATE[dt], (depth, err)


@pytest.mark.parametrize("dt", DTS)
def test_closed_forms_on_gpu(svlib, cuda_dev, dt):
    n = 13
    st = gpu_state(n, ghz_circuit(n), dt)
    ref = np.zeros(2 ** n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert maxabs(st, ref) < TOL_STATE[dt]
    x = 1234
    prep = [Gate("x", [q]) for q in range(n) if (x >> q) & 1]
    st = gpu_state(n, prep + qft_circuit(n), dt)
    ref = np.exp(2j * math.pi * x * np.arange(2 ** n) / 2 ** n) / math.sqrt(2 ** n)
    assert maxabs(st, ref) < TOL_STATE[dt]


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("n", [1, 4, 9, 10, 11, 12, 16])
def test_expectations(svlib, cuda_dev, dt, n):
    gates = random_circuit(n, 60, seed=n, max_controls=1, max_unitary_k=min(3, n))
    ref = oracle.run(n, gates)
    st = gpu_state(n, gates, dt)
    terms = random_pauli_terms(n, 40, seed=n + 5, max_weight=min(4, n))
    terms += [Term("Z", [q], 1.0) for q in range(n)] + [Term("X", [n - 1], 0.5)]
    got = B.sv_expect(st, terms)
    _, want = oracle.expect_terms(ref, n, terms)
    assert np.max(np.abs(got - want)) < TOL_EXPECT[dt]
    z = B.sv_expect_z_all(st)
    per, s = oracle.expect_z_all(ref, n)
    assert np.max(np.abs(z[:n] - per)) < TOL_EXPECT[dt]
    # sum_q <Z_q> is one expectation (of H = sum_q Z_q): the same bar, no factor n
    assert abs(z[n] - s) < TOL_EXPECT[dt]


def test_expectations_into_device_buffer(svlib, cuda_dev):
    import torch
    n = 14
    gates = random_circuit(n, 40, seed=2)
    st = gpu_state(n, gates, B.SV_C64)
    terms = random_pauli_terms(n, 20, seed=3)
    out = torch.zeros(len(terms), dtype=torch.float64, device="cuda")
    B.sv_expect(st, terms, out=out)
    zo = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    B.sv_expect_z_all(st, out=zo)
    torch.cuda.synchronize()
    assert np.allclose(out.cpu().numpy(), B.sv_expect(st, terms), atol=0, rtol=0)
    assert np.allclose(zo.cpu().numpy(), B.sv_expect_z_all(st), atol=0, rtol=0)


@pytest.mark.parametrize("dt", DTS)
def test_deterministic_bitwise(svlib, cuda_dev, dt):
    n = 16
    gates = random_circuit(n, 100, seed=9)
    a = gpu_state(n, gates, dt).cpu().numpy()
    b = gpu_state(n, gates, dt).cpu().numpy()
    assert np.array_equal(a, b)
    st = gpu_state(n, gates, dt)
    terms = random_pauli_terms(n, 10, seed=1)
    assert np.array_equal(B.sv_expect(st, terms), B.sv_expect(st, terms))


def test_parameter_slots_on_gpu(svlib, cuda_dev):
    n = 6
    gates = random_circuit(n, 50, seed=4, n_slots=7)
    params = np.random.default_rng(1).random(7) * 6
    ref = oracle.run(n, gates, params)
    st = gpu_state(n, gates, B.SV_C128, params=params)
    assert maxabs(st, ref) < 1e-12


def test_initial_state_and_inverse_restores(svlib, cuda_dev):
    n = 18
    rng = np.random.default_rng(0)
    v = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    v /= np.linalg.norm(v)
    gates = random_circuit(n, 80, seed=5, max_unitary_k=2)
    ref = oracle.run(n, gates, init=v)
    st = gpu_state(n, gates, B.SV_C128, init=v)
    assert maxabs(st, ref) < 1e-12


def test_boundary_rejects_bad_device_buffers(svlib, cuda_dev):
    import torch
    small = torch.zeros(2 ** 10, dtype=torch.complex64, device="cuda")
    import ctypes
    st = svlib.sv_init_basis(ctypes.c_void_p(small.data_ptr()), 30, B.SV_C64, 0, None)
    assert st == 1  # smaller than 2^30 amplitudes: refused before any launch
    st = svlib.sv_init_basis(ctypes.c_void_p(small.data_ptr() + 8), 4, B.SV_C64, 0, None)
    assert st == 1  # misaligned
    host = np.zeros(16, dtype=np.complex64)
    st = svlib.sv_init_basis(ctypes.c_void_p(host.ctypes.data), 4, B.SV_C64, 0, None)
    assert st == 1  # host memory
    # the library still works afterwards
    ok = torch.empty(16, dtype=torch.complex64, device="cuda")
    B.sv_init_basis(ok, 3)
    torch.cuda.synchronize()
    assert ok.cpu().numpy()[3] == 1


def test_run_host_end_to_end(svlib, cuda_dev):
    n = 16
    gates = fused_layered_u3_cz(n, 4, seed=1)
    ref = oracle.run(n, gates)
    out_state = np.zeros(2 ** n, dtype=np.complex128)
    z = B.sv_run_host(n, B.SV_C128, gates, fuse_max_k=5, state_out=out_state)
    assert np.max(np.abs(out_state - ref)) < 1e-12
    per, s = oracle.expect_z_all(ref, n)
    assert np.max(np.abs(z[:n] - per)) < 1e-11
    v = np.zeros(2 ** n, dtype=np.complex64)
    v[5] = 1
    z2 = B.sv_run_host(n, B.SV_C64, [], state_in=v)
    assert abs(z2[0] + 1) < 1e-6 and abs(z2[1] - 1) < 1e-6 and abs(z2[2] + 1) < 1e-6


def test_library_owned_state(svlib, cuda_dev):
    s = B.SvState(10, B.SV_C128)
    got = s.get()
    assert got[0] == 1 and np.count_nonzero(got) == 1
    v = (np.arange(1024) + 1j).astype(np.complex128)
    s.set(v)
    assert np.array_equal(s.get(), v)
    s.free()


def test_26q_c64_product_layers_then_cz_sampled_amplitudes(svlib, cuda_dev):
    """The 12-qubit-tile path (complex64 states of 26 qubits and more) against
    amplitudes the oracle computes one at a time: 12 layers of Haar-angle U3 on
    every qubit leave a product state (per qubit, the oracle's 2-vector), and
    a closing layer of CZ on even then odd neighbour pairs multiplies amplitude
    b by (-1)^(number of neighbour pairs with both bits set).  Closing phases
    cross passes and the CZs fold into tables on the way."""
    import torch
    n, layers = 26, 12
    rng = np.random.default_rng(26)
    gates = []
    for _ in range(layers):
        for q in range(n):
            gates.append(Gate("u3", [q], params=list(rng.uniform(0, 2 * np.pi, 3))))
    for start in (0, 1):
        for q in range(start, n - 1, 2):
            gates.append(Gate("z", [q + 1], controls=[q]))
    _, passes, _ = B.sv_plan_info(n, B.SV_C64, gates, fuse_max_k=5)
    assert passes >= 2
    st = torch.empty(2 ** n, dtype=torch.complex64, device="cuda")
    B.sv_init_basis(st, 0)
    B.sv_apply_circuit(st, gates, fuse_max_k=5)
    torch.cuda.synchronize()
    # per qubit: the oracle's one-qubit state after that qubit's gates
    vec = []
    for q in range(n):
        mine = [Gate("u3", [0], params=g.params) for g in gates if g.name == "u3" and g.targets == [q]]
        vec.append(oracle.run(1, mine))
    idx = rng.integers(0, 2 ** n, 2000, dtype=np.int64)
    got = st[torch.as_tensor(idx, device="cuda")].cpu().numpy().astype(np.complex128)
    for b, gv in zip(idx.tolist(), got):
        bits = [(b >> q) & 1 for q in range(n)]
        amp = complex(np.prod([vec[q][bits[q]] for q in range(n)]))
        if sum(bits[q] & bits[q + 1] for q in range(n - 1)) & 1:
            amp = -amp
        assert abs(gv - amp) <= TOL_STATE[B.SV_C64], (b, gv, amp)
    norm = float(torch.linalg.vector_norm(st.view(torch.float32).double()))
    assert abs(norm - 1) < 1e-4


@pytest.mark.slow
def test_full_size_30q_c64_forward_then_inverse(svlib, cuda_dev):
    """At the bench's size (30 qubits, 2^30 amplitudes) the oracle cannot run
    the circuit, so check properties that hold at any size: the norm stays 1,
    and the circuit followed by its exact inverse returns |0..0>."""
    import torch
    n = 30
    gates = fused_layered_u3_cz(n, 20, seed=0)
    inv = []
    for g in reversed(gates):
        if g.name == "u3":
            th, ph, la = g.params
            inv.append(Gate("u3", g.targets, params=[-th, -la, -ph]))
        else:
            inv.append(g)
    st = torch.empty(2 ** n, dtype=torch.complex64, device="cuda")
    B.sv_init_basis(st, 0)
    B.sv_apply_circuit(st, gates, fuse_max_k=5)
    norm = float(torch.linalg.vector_norm(st.view(torch.float32).double()))
    assert abs(norm - 1) < 1e-4
    B.sv_apply_circuit(st, inv, fuse_max_k=5)
    st[0] -= 1
    err = float(st.abs().max())
    assert err < 1e-4, err
