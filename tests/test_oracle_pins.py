"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here retypes the oracle's own formulas: each check reaches the same
quantity by another route (a closed form, a library routine such as expm or
the FFT, a brute-force Kronecker embedding, an algebraic identity between
gates, or an independent derivative), chosen so that a dropped term, a wrong
sign, a wrong bit index or a transposed operand in the oracle fails at least
one of them.
"""

import math

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from workloads import (Gate, Term, ghz_circuit, haar_unitary, hea_hamiltonian, hea_params, hea_ring,
                       layered_ry_rz_cnot, qft_circuit, random_circuit, random_pauli_terms)

# Textbook constants used only by the brute-force checks below.
I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
PAULI = {"I": I2, "X": PX, "Y": PY, "Z": PZ}


def M(name, *params):
    return oracle.gate_matrix(Gate(name, [0] if name not in ("swap", "rxx", "ryy", "rzz") else [0, 1],
                                   params=list(params)))


def unit(n, b):
    v = np.zeros(2 ** n, dtype=complex)
    v[b] = 1
    return v


def kron_chain(ops):
    """ops[q] acts on qubit q; qubit n-1 is the most significant factor."""
    out = np.array([[1.0 + 0j]])
    for op in reversed(ops):
        out = np.kron(out, op)
    return out


def full_matrix(n, U, targets, controls=(), cstates=()):
    """Brute-force 2^n x 2^n embedding of a (controlled) k-qubit matrix as a
    sum of Kronecker products of single-qubit matrix units and projectors."""
    d = U.shape[0]
    F = np.zeros((2 ** n, 2 ** n), dtype=complex)
    proj = [I2] * n
    for c, s in zip(controls, cstates):
        proj[c] = np.diag([1.0 - s, float(s)]).astype(complex)
    for r in range(d):
        for c in range(d):
            if U[r, c] == 0:
                continue
            ops = list(proj)
            for i, t in enumerate(targets):
                e = np.zeros((2, 2), dtype=complex)
                e[(r >> i) & 1, (c >> i) & 1] = 1
                ops[t] = e
            F += U[r, c] * kron_chain(ops)
    if controls:
        F += np.eye(2 ** n) - kron_chain(proj)
    return F


def brute_run(n, gates, params=None):
    psi = unit(n, 0)
    for g in gates:
        U = oracle.gate_matrix(g, params)
        psi = full_matrix(n, U, g.targets, g.controls, g.control_states) @ psi
    return psi


def dense_pauli(n, term):
    ops = [I2] * n
    for letter, q in zip(term.paulis, term.qubits):
        ops[q] = PAULI[letter]
    return kron_chain(ops)


# ------------------------------------------------------------ gate matrices

ONE_Q = ["i", "x", "y", "z", "h", "s", "sdg", "t", "tdg", "sx", "rx", "ry", "rz", "p", "u2", "u3"]


@pytest.mark.parametrize("name", ONE_Q + ["swap", "rxx", "ryy", "rzz"])
def test_every_gate_is_unitary(name):
    rng = np.random.default_rng(1)
    U = M(name, *(rng.random(3) * 2 * math.pi))
    assert np.allclose(U.conj().T @ U, np.eye(U.shape[0]), atol=1e-14)


def test_pauli_algebra():
    X, Y, Z = M("x"), M("y"), M("z")
    assert np.allclose(X @ Y, 1j * Z)
    assert np.allclose(Y @ Z, 1j * X)
    assert np.allclose(Z @ X, 1j * Y)
    # the gate's Y agrees with the Sec. 4.4 Pauli action (x = z = 1, nY = 1)
    for b in (0, 1):
        out = oracle.pauli_apply(unit(1, b), 1, [Term("Y", [0], 1.0)])
        assert np.allclose(out, Y @ unit(1, b))


def test_clifford_and_phase_identities():
    X, Y, Z, H = M("x"), M("y"), M("z"), M("h")
    S, T, Sdg, Tdg, SX = M("s"), M("t"), M("sdg"), M("tdg"), M("sx")
    assert np.allclose(H @ X @ H, Z)
    assert np.allclose(H @ Z @ H, X)
    assert np.allclose(H @ Y @ H, -Y)
    assert np.allclose(H @ unit(1, 0), np.array([1, 1]) / math.sqrt(2))
    assert np.allclose(S @ S, Z)
    assert np.allclose(T @ T, S)
    assert np.allclose(Sdg, S.conj().T)
    assert np.allclose(Tdg, T.conj().T)
    assert np.allclose(SX @ SX, X)
    assert np.allclose(S @ X @ Sdg, Y)


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.7, math.pi, 4.2])
def test_rotations_are_exponentials(theta):
    # R_P(theta) = exp(-i theta P / 2) (Sec. 9.1), by the matrix exponential
    for name, P in (("rx", PX), ("ry", PY), ("rz", PZ)):
        assert np.allclose(M(name, theta), expm(-0.5j * theta * P), atol=1e-14)
    for name, P in (("rxx", np.kron(PX, PX)), ("ryy", np.kron(PY, PY)), ("rzz", np.kron(PZ, PZ))):
        assert np.allclose(M(name, theta), expm(-0.5j * theta * P), atol=1e-14)
    # RZ = e^{-i theta/2} P(theta)
    assert np.allclose(M("rz", theta), np.exp(-0.5j * theta) * M("p", theta))


def test_rx_pi_is_minus_i_x():
    assert np.allclose(M("rx", math.pi), -1j * PX, atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_u3_euler_decomposition(seed):
    th, ph, la = np.random.default_rng(seed).random(3) * 2 * math.pi
    # U3(th, ph, la) = e^{i(ph+la)/2} RZ(ph) RY(th) RZ(la)
    rhs = np.exp(0.5j * (ph + la)) * M("rz", ph) @ M("ry", th) @ M("rz", la)
    assert np.allclose(M("u3", th, ph, la), rhs, atol=1e-14)
    assert np.allclose(M("u3", th, -math.pi / 2, math.pi / 2), M("rx", th), atol=1e-14)
    assert np.allclose(M("u3", th, 0, 0), M("ry", th), atol=1e-14)
    assert np.allclose(M("u3", 0, 0, la), M("p", la), atol=1e-14)
    assert np.allclose(M("u2", ph, la), M("u3", math.pi / 2, ph, la), atol=1e-14)


def test_swap_from_three_cnots():
    n = 2
    a = oracle.run(n, [Gate("swap", [0, 1])], init=None)
    assert np.allclose(a, unit(2, 0))
    for b in range(4):
        s = oracle.run(n, [Gate("swap", [0, 1])], init=unit(2, b))
        c = oracle.run(n, [Gate("x", [1], [0]), Gate("x", [0], [1]), Gate("x", [1], [0])], init=unit(2, b))
        assert np.allclose(s, c)
    assert np.allclose(oracle.run(2, [Gate("swap", [0, 1])], init=unit(2, 1)), unit(2, 2))


# ------------------------------------------------------------ application

def test_endianness_x_on_qubit_q_sets_bit_q():
    n = 5
    for q in range(n):
        psi = oracle.run(n, [Gate("x", [q])])
        assert np.allclose(psi, unit(n, 1 << q))


def test_two_qubit_matrix_bit_order():
    # targets[0] is the least-significant matrix bit: a matrix that maps
    # |j> -> |(j+1) mod 4> sends |b0=1,b1=0> (j=1) to j=2 (b1 set).
    P = np.roll(np.eye(4), 1, axis=0).astype(complex)
    psi = oracle.run(3, [Gate("unitary", [2, 0], matrix=P)], init=unit(3, 1 << 2))
    assert np.allclose(psi, unit(3, 1 << 0))


def test_ghz_closed_form():
    for n in (2, 5, 9):
        psi = oracle.run(n, ghz_circuit(n))
        ref = np.zeros(2 ** n, dtype=complex)
        ref[0] = ref[-1] = 1 / math.sqrt(2)
        assert np.allclose(psi, ref, atol=1e-15)


@pytest.mark.parametrize("n", [1, 3, 6, 10])
def test_qft_closed_form_and_fft(n):
    N = 2 ** n
    rng = np.random.default_rng(n)
    for x in rng.integers(0, N, size=3):
        prep = [Gate("x", [q]) for q in range(n) if (int(x) >> q) & 1]
        psi = oracle.run(n, prep + qft_circuit(n))
        y = np.arange(N)
        ref = np.exp(2j * math.pi * int(x) * y / N) / math.sqrt(N)
        assert np.allclose(psi, ref, atol=1e-12)
    # on an arbitrary input the QFT is sqrt(N) * inverse DFT (numpy's ifft)
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    v /= np.linalg.norm(v)
    out = oracle.run(n, qft_circuit(n), init=v)
    assert np.allclose(out, np.fft.ifft(v) * math.sqrt(N), atol=1e-12)


def test_qft_without_swaps_has_paper_gate_count():
    assert len(qft_circuit(16, with_swaps=False)) == 136


@pytest.mark.parametrize("seed", range(6))
def test_random_circuits_match_brute_force_kronecker(seed):
    n = 6
    gates = random_circuit(n, 40, seed=seed, max_controls=2, max_unitary_k=3)
    assert np.allclose(oracle.run(n, gates), brute_run(n, gates), atol=1e-12)


def test_layered_family_matches_brute_force_and_is_not_bit_reversal_invariant():
    n = 5
    gates = layered_ry_rz_cnot(n, 3, seed=3)
    psi = oracle.run(n, gates)
    assert np.allclose(psi, brute_run(n, gates), atol=1e-12)
    rev = np.array([int(format(b, "0%db" % n)[::-1], 2) for b in range(2 ** n)])
    assert not np.allclose(psi, psi[rev], atol=1e-3)


def test_control_state_zero_is_x_conjugated_control():
    n = 3
    rng = np.random.default_rng(0)
    U = haar_unitary(rng, 2, special=False)
    a = oracle.run(n, [Gate("h", [0]), Gate("h", [1]), Gate("unitary", [2], [0, 1], [0, 1], matrix=U)])
    b = oracle.run(n, [Gate("h", [0]), Gate("h", [1]), Gate("x", [0]),
                       Gate("unitary", [2], [0, 1], [1, 1], matrix=U), Gate("x", [0])])
    assert np.allclose(a, b, atol=1e-14)


def test_norm_preserved_and_inverse_restores():
    n = 8
    gates = random_circuit(n, 120, seed=11, max_controls=3, max_unitary_k=4)
    psi = oracle.run(n, gates)
    assert abs(np.linalg.norm(psi) - 1) < 1e-13
    inv = []
    for g in reversed(gates):
        U = oracle.gate_matrix(g)
        inv.append(Gate("unitary", list(g.targets), list(g.controls), list(g.control_states),
                        matrix=U.conj().T))
    back = oracle.run(n, inv, init=psi)
    assert np.allclose(back, unit(n, 0), atol=1e-12)


def test_parameter_slots_bind_and_unbound_raises():
    g = [Gate("ry", [0], params=[0.0], slots=[1])]
    psi = oracle.run(1, g, param_values=[0.0, math.pi])
    assert np.allclose(psi, unit(1, 1), atol=1e-15)
    with pytest.raises(ValueError):
        oracle.run(1, g, param_values=None)


# ------------------------------------------------------------ expectations

@pytest.mark.parametrize("theta", [0.2, 1.1, 2.9, 5.0])
def test_single_qubit_expectation_closed_forms(theta):
    psi = oracle.run(1, [Gate("ry", [0], params=[theta])])
    e = lambda s: oracle.expect_terms(psi, 1, [Term(s, [0], 1.0)])[0]
    assert abs(e("Z") - math.cos(theta)) < 1e-14
    assert abs(e("X") - math.sin(theta)) < 1e-14
    assert abs(e("Y")) < 1e-14
    psi = oracle.run(1, [Gate("rx", [0], params=[theta])])
    assert abs(oracle.expect_terms(psi, 1, [Term("Y", [0], 1.0)])[0] + math.sin(theta)) < 1e-14


def test_ghz_expectations():
    n = 6
    psi = oracle.run(n, ghz_circuit(n))
    per, s = oracle.expect_z_all(psi, n)
    assert np.allclose(per, 0, atol=1e-15) and abs(s) < 1e-14
    assert abs(oracle.expect_terms(psi, n, [Term("ZZ", [1, 4], 1.0)])[0] - 1) < 1e-14
    assert abs(oracle.expect_terms(psi, n, [Term("X" * n, list(range(n)), 1.0)])[0] - 1) < 1e-14
    psi2 = oracle.run(2, ghz_circuit(2))
    assert abs(oracle.expect_terms(psi2, 2, [Term("YY", [0, 1], 1.0)])[0] + 1) < 1e-14


@pytest.mark.parametrize("seed", range(4))
def test_pauli_expectations_match_dense_kronecker(seed):
    n = 6
    psi = oracle.run(n, random_circuit(n, 50, seed=seed))
    terms = random_pauli_terms(n, 12, seed=seed + 100)
    tot, per = oracle.expect_terms(psi, n, terms)
    ref = [np.vdot(psi, dense_pauli(n, t) @ psi).real for t in terms]
    assert np.allclose(per, ref, atol=1e-13)
    assert abs(tot - sum(t.coeff * r for t, r in zip(terms, ref))) < 1e-12
    Hpsi = oracle.pauli_apply(psi, n, terms)
    Hd = sum(t.coeff * dense_pauli(n, t) for t in terms)
    assert np.allclose(Hpsi, Hd @ psi, atol=1e-12)


def test_sum_z_equals_probability_weighted_popcount():
    n = 7
    psi = oracle.run(n, random_circuit(n, 60, seed=5))
    per, s = oracle.expect_z_all(psi, n)
    p = np.abs(psi) ** 2
    pop = np.array([bin(b).count("1") for b in range(2 ** n)])
    assert abs(s - float(np.sum(p * (n - 2 * pop)))) < 1e-13
    for i in range(n):
        bit = (np.arange(2 ** n) >> i) & 1
        assert abs(per[i] - float(np.sum(p * (1 - 2 * bit)))) < 1e-13


# ------------------------------------------------------------ gradients

@pytest.mark.parametrize("theta", [0.4, 2.0, 3.7])
def test_adjoint_single_rotation_closed_form(theta):
    g = [Gate("ry", [0], params=[0.0], slots=[0])]
    val, grad = oracle.adjoint_grad(1, g, [theta], [Term("Z", [0], 1.0)], 1)
    assert abs(val - math.cos(theta)) < 1e-14
    assert abs(grad[0] + math.sin(theta)) < 1e-14


def test_adjoint_matches_parameter_shift_and_fd_on_hea():
    n, layers = 5, 3
    gates = hea_ring(n, layers)
    terms = hea_hamiltonian(n, 0.7)
    P = 2 * n * layers
    theta = hea_params(1, P, seed=7)[0]
    val, g_adj = oracle.adjoint_grad(n, gates, theta, terms, P)
    assert abs(val - oracle.energy(n, gates, theta, terms)) < 1e-13
    g_ps = oracle.param_shift_grad(n, gates, theta, terms, P)
    g_fd = oracle.fd_grad(n, gates, theta, terms, P, h=1e-3)
    assert np.max(np.abs(g_adj - g_ps)) < 1e-11
    assert np.max(np.abs(g_adj - g_fd)) < 5e-6  # O(h^2)


def test_adjoint_shared_slots_controlled_rotations_and_phase_vs_fd():
    n = 4
    rng = np.random.default_rng(3)
    gates = [Gate("h", [q]) for q in range(n)]
    gates += [Gate("rx", [0], params=[0], slots=[0]), Gate("rzz", [1, 3], params=[0], slots=[1]),
              Gate("ry", [2], [0], [0], params=[0], slots=[2]), Gate("p", [3], [1], params=[0], slots=[0]),
              Gate("ryy", [0, 2], params=[0], slots=[3]), Gate("rx", [1], params=[0], slots=[2]),
              Gate("x", [2], [3]), Gate("rz", [2], params=[0], slots=[3])]
    terms = random_pauli_terms(n, 6, seed=9)
    theta = rng.random(4) * 2 * math.pi
    _, g_adj = oracle.adjoint_grad(n, gates, theta, terms, 4)
    g_fd = oracle.fd_grad(n, gates, theta, terms, 4, h=1e-4)
    assert np.max(np.abs(g_adj - g_fd)) < 1e-7


def test_adjoint_rejects_slot_on_gate_without_generator():
    with pytest.raises(ValueError):
        oracle.adjoint_grad(1, [Gate("u3", [0], params=[0, 0, 0], slots=[0, -1, -1])], [0.1],
                            [Term("Z", [0], 1.0)], 1)


# ------------------------------------------------------------ fusion

@pytest.mark.parametrize("kmax", [2, 3, 4, 5])
def test_fused_equals_unfused(kmax):
    n = 8
    gates = random_circuit(n, 80, seed=kmax, max_controls=1, max_unitary_k=2)
    blocks = oracle.fuse(n, gates, kmax)
    assert blocks[0][0] == 0 and blocks[-1][1] == len(gates)
    fused = [Gate("unitary", qs, matrix=m) for (_, _, qs, m) in blocks]
    for (a, b, qs, _) in blocks:
        width = len(set(q for g in gates[a:b] for g_q in [g.qubits()] for q in g_q))
        assert width == len(qs)
        assert len(qs) <= kmax or b - a == 1
    a = oracle.run(n, gates)
    b = oracle.run(n, fused)
    # the paper's fused/unfused overlap check is 1 +- 1e-8 (Sec. 9.2)
    assert abs(abs(np.vdot(a, b)) - 1) < 1e-12
    assert np.allclose(a, b, atol=1e-12)


def test_fusion_block_boundaries_on_a_known_sequence():
    g = [Gate("h", [q]) for q in range(4)] + [Gate("x", [1], [0]), Gate("x", [3], [2])]
    blocks = oracle.fuse(4, g, 2)
    assert [(a, b) for a, b, _, _ in blocks] == [(0, 2), (2, 4), (4, 5), (5, 6)]
    blocks = oracle.fuse(4, g, 4)
    assert [(a, b) for a, b, _, _ in blocks] == [(0, 6)]
    # no reordering: H0 X1 H0 with k=1 stays three blocks
    g2 = [Gate("h", [0]), Gate("x", [1]), Gate("h", [0])]
    assert len(oracle.fuse(2, g2, 1)) == 3


# ---------------------------------------------------------------- excitation gates
# Single and double excitation (Sec. 4.2 gate table): a rotation by theta/2
# between the two basis states that exchange the excitation(s), identity on
# every other state; generator spectrum {-1, 0, 1} (four-term shift rule).

def _basis(n, bits):
    psi = np.zeros(2 ** n, complex)
    psi[sum(1 << q for q in bits)] = 1.0
    return psi


def test_exc1_rotates_the_exchanged_pair():
    from workloads import Gate
    n, th = 4, 0.83
    c, s = np.cos(th / 2), np.sin(th / 2)
    out = oracle.run(n, [Gate("exc1", [1, 3], params=[th])], init=_basis(n, [1]))  # |t0 t1> = |10>
    want = c * _basis(n, [1]) + s * _basis(n, [3])
    assert np.abs(out - want).max() < 1e-15
    for occ in ([], [1, 3], [0, 2]):  # |00>, |11> and spectators: unchanged
        assert np.abs(oracle.run(n, [Gate("exc1", [1, 3], params=[th])], init=_basis(n, occ)) - _basis(n, occ)).max() == 0


def test_exc2_rotates_the_exchanged_pair():
    from workloads import Gate
    n, th = 5, -1.37
    c, s = np.cos(th / 2), np.sin(th / 2)
    t = [4, 0, 3, 1]
    out = oracle.run(n, [Gate("exc2", t, params=[th])], init=_basis(n, [4, 0]))
    assert np.abs(out - (c * _basis(n, [4, 0]) + s * _basis(n, [3, 1]))).max() < 1e-15
    out = oracle.run(n, [Gate("exc2", t, params=[th])], init=_basis(n, [3, 1]))
    assert np.abs(out - (-s * _basis(n, [4, 0]) + c * _basis(n, [3, 1]))).max() < 1e-15
    assert np.abs(oracle.run(n, [Gate("exc2", t, params=[th])], init=_basis(n, [4, 3])) - _basis(n, [4, 3])).max() == 0


def test_excitations_conserve_the_number_of_ones():
    from workloads import Gate
    rng = np.random.default_rng(4)
    n = 7
    gates = []
    for _ in range(40):
        q = [int(x) for x in rng.permutation(n)[:4]]
        gates.append(Gate("exc1", q[:2], params=[rng.uniform(0, 6.3)]) if rng.random() < 0.5
                     else Gate("exc2", q, params=[rng.uniform(0, 6.3)]))
    out = oracle.run(n, gates, init=_basis(n, [0, 2, 5]))
    weights = np.array([bin(i).count("1") for i in range(2 ** n)])
    assert np.abs(out[weights != 3]).max() < 1e-14
    assert abs(np.linalg.norm(out) - 1) < 1e-13


def test_excitation_gradients_four_term_rule_fd_and_adjoint_agree():
    from workloads import Gate, Term
    n = 6
    gates = random_circuit(n, 25, seed=8) + [Gate("exc1", [1, 3], slots=[0]), Gate("ry", [2], slots=[1]),
                                             Gate("exc2", [0, 2, 4, 5], slots=[2]), Gate("exc1", [4, 0], slots=[3])]
    pv = np.array([0.3, 1.1, -0.7, 2.0])
    H = [Term("ZZ", [0, 1], 0.6), Term("X", [3], 0.4), Term("YZ", [2, 5], -0.8)]
    _, adj = oracle.adjoint_grad(n, gates, pv, H, 4)
    shift = oracle.param_shift_grad(n, gates, pv, H, 4)
    fd = oracle.fd_grad(n, gates, pv, H, 4)
    assert np.abs(shift - adj).max() < 1e-12  # the four-term rule is exact
    assert np.abs(fd - adj).max() < 1e-6      # O(h^2), h = 1e-3
