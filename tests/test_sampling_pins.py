"""Pins of the oracle's measurement (Sec. 5.3: p_i = x_i^2 + y_i^2, normalised;
finite-shot draws of basis indices from it), against what the mathematics
fixes: closed-form distributions, an exact quantile bound and invariants."""
import numpy as np
import pytest

import oracle
from workloads import ghz_circuit, random_circuit


def test_probabilities_are_squared_moduli_and_normalised():
    n = 9
    psi = oracle.run(n, random_circuit(n, 80, seed=4))
    p = oracle.probabilities(psi * 1.7, n, normalise=False)
    assert np.allclose(p, np.abs(psi * 1.7) ** 2, rtol=1e-15, atol=0)
    q = oracle.probabilities(psi * 1.7, n, normalise=True)
    assert abs(q.sum() - 1.0) < 1e-14
    assert np.allclose(q, np.abs(psi) ** 2, rtol=1e-13, atol=1e-18)


@pytest.mark.parametrize("n,k", [(5, 0), (5, 31), (8, 77), (12, 4095)])
def test_basis_state_always_gives_its_index(n, k):
    psi = np.zeros(2 ** n, complex)
    psi[k] = np.exp(0.3j)
    u = np.concatenate([np.random.default_rng(k).random(200), [0.0, 1.0 - 2.0 ** -53]])
    assert (oracle.sample(psi, n, u) == k).all()


@pytest.mark.parametrize("n", [5, 9, 14])
def test_uniform_superposition_is_floor_u_2n(n):
    psi = np.full(2 ** n, 2.0 ** (-n / 2), complex)  # every p_i = 2^-n exactly
    u = np.random.default_rng(n).random(5000)
    assert (oracle.sample(psi, n, u) == np.floor(u * 2 ** n).astype(np.uint64)).all()


def test_ghz_splits_at_one_half():
    n = 10
    psi = oracle.run(n, ghz_circuit(n))
    u = np.array([0.0, 0.25, 0.5 - 2.0 ** -53, 0.5, 0.75, 1.0 - 2.0 ** -53])
    got = oracle.sample(psi, n, u)
    top = 2 ** n - 1
    # |psi_0|^2 and |psi_top|^2 round to the same double, so the split is exact
    assert (got == np.array([0, 0, 0, top, top, top], dtype=np.uint64)).all()


def test_quantile_grid_matches_probabilities():
    # u_k = (k + 1/2) / K: index i is drawn for the grid points inside
    # [F_{i-1}, F_i), so its count differs from p_i K by at most 1 (plus the
    # 2^-61 quantisation of each p_i)
    n, K = 7, 1 << 16
    psi = oracle.run(n, random_circuit(n, 60, seed=9))
    p = np.abs(psi) ** 2
    u = (np.arange(K) + 0.5) / K
    cnt = np.bincount(oracle.sample(psi, n, u).astype(np.int64), minlength=2 ** n)
    assert cnt.sum() == K
    assert np.abs(cnt - p / p.sum() * K).max() <= 1.0 + 1e-6


def test_zero_amplitudes_are_never_drawn():
    n = 8
    psi = oracle.run(n, random_circuit(n, 40, seed=2))
    psi[::3] = 0.0
    got = oracle.sample(psi, n, np.random.default_rng(0).random(20000))
    assert (got % 3 != 0).all()
