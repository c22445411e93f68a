"""Seeded gate-list, Hamiltonian and arrival-stream generators.

Every generator takes an explicit seed and draws from
``numpy.random.Generator(PCG64(seed))``; the same seed gives the same records
on every machine.  Records are plain data (see ``Gate`` and ``Term``); nothing
here computes a gate matrix from an angle.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

TWO_PI = 2.0 * math.pi

# Gate names understood by both the oracle and the CUDA library, with the
# number of targets and the number of angle parameters each takes.  The
# families follow the built-in gate table of Sec. 4.2.
GATE_ARITY = {
    "i": (1, 0), "x": (1, 0), "y": (1, 0), "z": (1, 0), "h": (1, 0),
    "s": (1, 0), "sdg": (1, 0), "t": (1, 0), "tdg": (1, 0), "sx": (1, 0),
    "rx": (1, 1), "ry": (1, 1), "rz": (1, 1), "p": (1, 1),
    "u2": (1, 2), "u3": (1, 3),
    "swap": (2, 0), "rxx": (2, 1), "ryy": (2, 1), "rzz": (2, 1),
    "unitary": (None, 0), "exc1": (2, 1), "exc2": (4, 1),
}


@dataclass
class Gate:
    """One circuit operation as the paper states it (Sec. 4.2, App. A.2).

    name:     lower-case gate family name (keys of ``GATE_ARITY``)
    targets:  target qubits; for a multi-qubit matrix targets[0] is the least
              significant bit of the matrix row/column index
    controls: control qubits (after the targets, as in the paper's API)
    control_states: per control, the basis state (0 or 1) that enables the gate
    params:   angle values (radians); ignored entries for parameter-free gates
    slots:    per angle, the index of a shared parameter vector entry that
              supplies the angle at run time, or -1 for the literal in params
    matrix:   for ``unitary`` only: a (2^k, 2^k) complex128 array
    """

    name: str
    targets: List[int]
    controls: List[int] = field(default_factory=list)
    control_states: List[int] = field(default_factory=list)
    params: List[float] = field(default_factory=list)
    slots: List[int] = field(default_factory=list)
    matrix: Optional[np.ndarray] = None

    def __post_init__(self):
        if not self.control_states:
            self.control_states = [1] * len(self.controls)
        nparam = GATE_ARITY[self.name][1]
        if len(self.params) < nparam:
            self.params = list(self.params) + [0.0] * (nparam - len(self.params))
        if not self.slots:
            self.slots = [-1] * len(self.params)

    def qubits(self) -> List[int]:
        return list(self.targets) + list(self.controls)


@dataclass
class Term:
    """A weighted Pauli string, e.g. Term("ZZ", [0, 3], -1.0) (Sec. 4.2)."""

    paulis: str
    qubits: List[int]
    coeff: float


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def haar_u3_angles(rng: np.random.Generator) -> Tuple[float, float, float]:
    """Euler angles (theta, phi, lambda) of a Haar-random SU(2) element.

    In the ZYZ parametrisation the Haar density is proportional to
    sin(theta) on [0, pi], so cos(theta) is uniform; phi and lambda are
    uniform on [0, 2 pi).
    """
    u = rng.random()
    theta = math.acos(1.0 - 2.0 * u)
    phi = rng.random() * TWO_PI
    lam = rng.random() * TWO_PI
    return theta, phi, lam


def haar_unitary(rng: np.random.Generator, dim: int, special: bool = True) -> np.ndarray:
    """Haar-random dim x dim unitary (complex Ginibre + QR with phase fix).

    The phases of R's diagonal are folded into Q so that the distribution is
    Haar (Mezzadri, 2007); with ``special`` the result is scaled by
    det^(-1/dim) to land in SU(dim).
    """
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    q = q * (d / np.abs(d))[np.newaxis, :]
    if special:
        det = np.linalg.det(q)
        q = q * (det ** (-1.0 / dim))
    return np.ascontiguousarray(q, dtype=np.complex128)


# ---------------------------------------------------------------- workloads

def layered_ry_rz_cnot(n: int = 12, layers: int = 10, seed: int = 0) -> List[Gate]:
    """Layered ansatz: per layer RY then RZ on every qubit, then a CNOT ladder.

    Angles are uniform in [0, 2 pi).  The CNOT ladder is i -> i+1 for
    i = 0..n-2 (control i, target i+1).
    """
    rng = _rng(seed)
    gates: List[Gate] = []
    for _ in range(layers):
        for q in range(n):
            gates.append(Gate("ry", [q], params=[rng.random() * TWO_PI]))
            gates.append(Gate("rz", [q], params=[rng.random() * TWO_PI]))
        for q in range(n - 1):
            gates.append(Gate("x", [q + 1], controls=[q]))
    return gates


def fused_layered_u3_cz(n: int = 30, layers: int = 20, seed: int = 0) -> List[Gate]:
    """Per layer: Haar-angle U3 on every qubit, CZ on (0,1),(2,3),..., then on
    (1,2),(3,4),...  (59 gates per layer at n = 30)."""
    rng = _rng(seed)
    gates: List[Gate] = []
    for _ in range(layers):
        for q in range(n):
            gates.append(Gate("u3", [q], params=list(haar_u3_angles(rng))))
        for q in range(0, n - 1, 2):
            gates.append(Gate("z", [q + 1], controls=[q]))
        for q in range(1, n - 1, 2):
            gates.append(Gate("z", [q + 1], controls=[q]))
    return gates


def precision_sweep(n: int = 24, n1: int = 400, n2: int = 200, seed: int = 0) -> List[Gate]:
    """n1 Haar-random U(2) gates on uniform qubits and n2 Haar SU(4) gates on
    uniformly drawn ordered pairs of distinct qubits, interleaved by a seeded
    shuffle.  Matrices are explicit ``unitary`` records."""
    rng = _rng(seed)
    kinds = np.array([1] * n1 + [2] * n2)
    rng.shuffle(kinds)
    gates: List[Gate] = []
    for k in kinds:
        if k == 1:
            q = int(rng.integers(0, n))
            gates.append(Gate("unitary", [q], matrix=haar_unitary(rng, 2, special=False)))
        else:
            a = int(rng.integers(0, n))
            b = int(rng.integers(0, n - 1))
            if b >= a:
                b += 1
            gates.append(Gate("unitary", [a, b], matrix=haar_unitary(rng, 4, special=True)))
    return gates


def hea_ring(n: int = 20, layers: int = 10) -> List[Gate]:
    """Hardware-efficient ansatz template with parameter slots.

    Per layer: RY then RZ on every qubit, then the CNOT ring i -> (i+1) mod n.
    Slots are numbered layer-major, then qubit, then (RY, RZ): the paper binds
    parameters in first-use order (Sec. 4.2).
    """
    gates: List[Gate] = []
    for layer in range(layers):
        for q in range(n):
            base = 2 * (layer * n + q)
            gates.append(Gate("ry", [q], params=[0.0], slots=[base]))
            gates.append(Gate("rz", [q], params=[0.0], slots=[base + 1]))
        for q in range(n):
            gates.append(Gate("x", [(q + 1) % n], controls=[q]))
    return gates


def hea_hamiltonian(n: int = 20, x_coeff: float = 0.7) -> List[Term]:
    """H = sum_i Z_i Z_{i+1 mod n} + x_coeff * sum_i X_i (periodic)."""
    terms = [Term("ZZ", [i, (i + 1) % n], 1.0) for i in range(n)]
    terms += [Term("X", [i], x_coeff) for i in range(n)]
    return terms


def hea_params(batch: int, n_params: int, seed: int = 0) -> np.ndarray:
    """(batch, n_params) float64 angles, uniform in [0, 2 pi)."""
    return _rng(seed).random((batch, n_params)) * TWO_PI


def serving_angles(n: int, depth: int, seed: int) -> np.ndarray:
    """(depth, n, 3) Haar-distributed U3 angles (theta, phi, lambda) of one
    serving request, drawn at once from ``seed`` (see ``haar_u3_angles``)."""
    u = _rng(seed).random((depth, n, 3))
    ang = np.empty_like(u)
    ang[..., 0] = np.arccos(1.0 - 2.0 * u[..., 0])
    ang[..., 1] = u[..., 1] * TWO_PI
    ang[..., 2] = u[..., 2] * TWO_PI
    return ang


def serving_circuit(n: int, depth: int, seed: int) -> List[Gate]:
    """One serving request: ``depth`` layers of Haar-angle U3 on all qubits
    followed by the CNOT ladder i -> i+1; angles from ``serving_angles``."""
    ang = serving_angles(n, depth, seed)
    gates: List[Gate] = []
    for d in range(depth):
        for q in range(n):
            gates.append(Gate("u3", [q], params=[float(x) for x in ang[d, q]]))
        for q in range(n - 1):
            gates.append(Gate("x", [q + 1], controls=[q]))
    return gates


def serving_stream(rate: float = 2000.0, duration: float = 60.0, n_lo: int = 8, n_hi: int = 26,
                   d_lo: int = 5, d_hi: int = 40, seed: int = 0, max_requests: Optional[int] = None):
    """Poisson arrivals: returns a list of (arrival_s, n_qubits, depth, circuit_seed).

    Inter-arrival times are exponential with mean 1/rate; n and depth are
    uniform on the closed ranges.  Circuits are drawn lazily from
    ``circuit_seed`` with ``serving_circuit`` so a long stream stays small.
    """
    rng = _rng(seed)
    out = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        n = int(rng.integers(n_lo, n_hi + 1))
        d = int(rng.integers(d_lo, d_hi + 1))
        cs = int(rng.integers(0, 2**62))
        out.append((t, n, d, cs))
        if max_requests is not None and len(out) >= max_requests:
            break
    return out


def ghz_circuit(n: int) -> List[Gate]:
    """H on qubit 0, then CNOT i -> i+1."""
    gates = [Gate("h", [0])]
    for q in range(n - 1):
        gates.append(Gate("x", [q + 1], controls=[q]))
    return gates


def qft_circuit(n: int, with_swaps: bool = True) -> List[Gate]:
    """Textbook QFT on a little-endian register (qubit n-1 is the most
    significant bit): for j = n-1 .. 0, H on j then controlled phases
    pi / 2^(j-m) from each m < j; then SWAP(i, n-1-i) when ``with_swaps``.
    Without the swaps it has n(n+1)/2 gates (136 at n = 16, Sec. 9.1)."""
    gates: List[Gate] = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate("h", [j]))
        for m in range(j - 1, -1, -1):
            gates.append(Gate("p", [j], controls=[m], params=[math.pi / (2 ** (j - m))]))
    if with_swaps:
        for i in range(n // 2):
            gates.append(Gate("swap", [i, n - 1 - i]))
    return gates


_ONE_Q = ["i", "x", "y", "z", "h", "s", "sdg", "t", "tdg", "sx", "rx", "ry", "rz", "p", "u2", "u3"]
_TWO_Q = ["swap", "rxx", "ryy", "rzz"]


def random_circuit(n: int, n_gates: int, seed: int = 0, max_controls: int = 2,
                   max_unitary_k: int = 3, families: Optional[Sequence[str]] = None,
                   n_slots: int = 0) -> List[Gate]:
    """Random gates over every family, with random controls and control states.

    Used by the parity tests to reach every code path: each gate picks a
    family, distinct random qubits for targets and controls (when n allows),
    angles uniform in [0, 2 pi) and, if ``n_slots`` > 0, binds each angle of
    a rotation to a random slot with probability 1/2.
    """
    rng = _rng(seed)
    fams = list(families) if families else _ONE_Q + _TWO_Q + ["unitary"]
    gates: List[Gate] = []
    for _ in range(n_gates):
        name = fams[int(rng.integers(0, len(fams)))]
        if name == "unitary":
            k = int(rng.integers(1, min(max_unitary_k, n) + 1))
        else:
            k = GATE_ARITY[name][0]
        if k > n:
            name, k = "h", 1
        nc = int(rng.integers(0, max_controls + 1)) if n - k > 0 else 0
        nc = min(nc, n - k)
        qs = [int(v) for v in rng.permutation(n)[: k + nc]]
        targets, controls = qs[:k], qs[k:]
        states = [int(v) for v in rng.integers(0, 2, size=nc)]
        nparam = GATE_ARITY[name][1]
        params = [float(v) for v in rng.random(nparam) * TWO_PI]
        slots = [-1] * nparam
        if n_slots > 0:
            for j in range(nparam):
                if rng.random() < 0.5:
                    slots[j] = int(rng.integers(0, n_slots))
        mat = haar_unitary(rng, 2 ** k, special=False) if name == "unitary" else None
        gates.append(Gate(name, targets, controls, states, params, slots, mat))
    return gates


def random_pauli_terms(n: int, n_terms: int, seed: int = 0, max_weight: int = 4) -> List[Term]:
    """Random weighted Pauli strings with letters from {X, Y, Z}."""
    rng = _rng(seed)
    terms: List[Term] = []
    for _ in range(n_terms):
        w = int(rng.integers(1, min(max_weight, n) + 1))
        qs = [int(v) for v in rng.permutation(n)[:w]]
        letters = "".join("XYZ"[int(v)] for v in rng.integers(0, 3, size=w))
        terms.append(Term(letters, qs, float(rng.standard_normal())))
    return terms
