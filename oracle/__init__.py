"""Plain complex128 CPU oracle for the state-vector hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may call it; the product package never imports it and
shares no code with it.  The arithmetic lives in ``sv_oracle.c`` (plain C99
``double complex``), compiled on first use with gcc; this module only converts
the seeded records of ``workloads`` into the oracle's own C structs and adds
the two gradient checks that need nothing but the forward oracle:

* the parameter-shift rule, df/dtheta = (f(theta + pi/2) - f(theta - pi/2)) / 2
  for each occurrence of a Pauli rotation (Sec. 4.2, shift-rule equation), and
* central finite differences (f(theta + h) - f(theta - h)) / (2 h) with
  h = 1e-3 (an independent numeric check, Sec. 7.3).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (closed forms, brute-force Kronecker unitaries,
gate identities, shift-rule / finite-difference agreement, fused == unfused).
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

MAXQ = 10

KINDS = {
    "i": 0, "x": 1, "y": 2, "z": 3, "h": 4, "s": 5, "sdg": 6, "t": 7, "tdg": 8, "sx": 9,
    "rx": 10, "ry": 11, "rz": 12, "p": 13, "u2": 14, "u3": 15,
    "swap": 16, "rxx": 17, "ryy": 18, "rzz": 19, "unitary": 20,
    "exc1": 21, "exc2": 22,
}
ROTATIONS = {"rx", "ry", "rz", "p", "rxx", "ryy", "rzz", "exc1", "exc2"}
EXCITATIONS = {"exc1", "exc2"}  # generators with spectrum {-1, 0, 1}: four-term shift rule


class OGGate(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("nt", ctypes.c_int32),
        ("t", ctypes.c_int32 * MAXQ),
        ("nc", ctypes.c_int32),
        ("c", ctypes.c_int32 * MAXQ),
        ("cstate", ctypes.c_int32 * MAXQ),
        ("p", ctypes.c_double * 3),
        ("slot", ctypes.c_int32),
        ("mat", ctypes.POINTER(ctypes.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compile ``sv_oracle.c`` into ``_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu99", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC,
               "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        cd = ctypes.c_double
        L.og_gate_matrix.argtypes = [P(OGGate), P(cd)]
        L.og_gate_matrix.restype = ctypes.c_int
        L.og_apply_circuit.argtypes = [ctypes.c_void_p, ctypes.c_int, P(OGGate), ctypes.c_int]
        L.og_apply_circuit.restype = ctypes.c_int
        L.og_zero_state.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.og_pauli_apply_add.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                         cd, ctypes.c_void_p]
        L.og_expect_pauli.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
        L.og_expect_pauli.restype = cd
        L.og_expect_z_all.argtypes = [ctypes.c_void_p, ctypes.c_int, P(cd), P(cd)]
        L.og_probabilities.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, P(cd)]
        L.og_probabilities.restype = None
        L.og_sample.argtypes = [ctypes.c_void_p, ctypes.c_int, P(cd), ctypes.c_int64, P(ctypes.c_uint64)]
        L.og_sample.restype = ctypes.c_int
        L.og_inner.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, P(cd), P(cd)]
        L.og_adjoint_grad.argtypes = [ctypes.c_int, P(OGGate), ctypes.c_int, P(ctypes.c_uint64),
                                      P(ctypes.c_uint64), P(cd), ctypes.c_int, P(cd), ctypes.c_int, P(cd)]
        L.og_adjoint_grad.restype = ctypes.c_int
        L.og_fuse.argtypes = [ctypes.c_int, P(OGGate), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int), P(cd), ctypes.c_int]
        L.og_fuse.restype = ctypes.c_int
        L.og_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def n_threads() -> int:
    return int(lib().og_num_threads())


# ---------------------------------------------------------------- records

class _Packed:
    """ctypes array of OGGate plus the matrix buffers it points into."""

    def __init__(self, gates, param_values: Optional[Sequence[float]]):
        self.keep = []
        self.arr = (OGGate * max(1, len(gates)))()
        for i, g in enumerate(gates):
            o = self.arr[i]
            o.kind = KINDS[g.name]
            o.nt = len(g.targets)
            o.nc = len(g.controls)
            if o.nt + o.nc > MAXQ:
                raise ValueError("oracle gate wider than %d qubits" % MAXQ)
            for j, q in enumerate(g.targets):
                o.t[j] = q
            for j, q in enumerate(g.controls):
                o.c[j] = q
                o.cstate[j] = int(g.control_states[j])
            vals = list(g.params) + [0.0] * (3 - len(g.params))
            for j, s in enumerate(g.slots):
                if s >= 0:
                    if param_values is None or s >= len(param_values):
                        raise ValueError("gate %d: parameter slot %d is unbound" % (i, s))
                    vals[j] = float(param_values[s])
            for j in range(3):
                o.p[j] = vals[j]
            o.slot = int(g.slots[0]) if (g.slots and g.name in ROTATIONS) else -1
            if g.slots and any(s >= 0 for s in g.slots) and g.name not in ROTATIONS:
                o.slot = -2  # bound to a slot but without a rotation generator
            if g.name == "unitary":
                m = np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128))
                if m.shape != (2 ** o.nt, 2 ** o.nt):
                    raise ValueError("unitary matrix shape does not match its targets")
                buf = np.ascontiguousarray(m.view(np.float64).reshape(-1))
                self.keep.append(buf)
                o.mat = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.n = len(gates)


def pauli_masks(terms) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(x_mask, z_mask, coeff) arrays: X sets x, Z sets z, Y sets both."""
    xs = np.zeros(len(terms), dtype=np.uint64)
    zs = np.zeros(len(terms), dtype=np.uint64)
    cs = np.zeros(len(terms), dtype=np.float64)
    for j, t in enumerate(terms):
        x = z = 0
        for letter, q in zip(t.paulis, t.qubits):
            b = 1 << q
            if letter in "XY":
                x |= b
            if letter in "ZY":
                z |= b
            if letter not in "IXYZ":
                raise ValueError("bad Pauli letter %r" % letter)
        xs[j], zs[j], cs[j] = x, z, t.coeff
    return xs, zs, cs


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------- calls

def gate_matrix(gate, param_values=None) -> np.ndarray:
    pk = _Packed([gate], param_values)
    out = np.zeros(2 * 1024, dtype=np.float64)
    d = lib().og_gate_matrix(pk.arr, _dp(out))
    if d == 0:
        raise ValueError("unknown gate kind")
    return out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()


def run(n: int, gates, param_values=None, init: Optional[np.ndarray] = None) -> np.ndarray:
    """psi = U_N ... U_1 |init> (|0..0> by default), complex128."""
    if init is None:
        psi = np.zeros(2 ** n, dtype=np.complex128)
        psi[0] = 1.0
    else:
        psi = np.array(init, dtype=np.complex128, copy=True)
        assert psi.shape == (2 ** n,)
    pk = _Packed(gates, param_values)
    rc = lib().og_apply_circuit(_ptr(psi), n, pk.arr, pk.n)
    if rc != 0:
        raise ValueError("oracle rejected gate %d" % (-rc - 1))
    return psi


def expect_terms(psi: np.ndarray, n: int, terms) -> Tuple[float, np.ndarray]:
    """(sum_j c_j <P_j>, array of <P_j>) for real coefficients c_j."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    xs, zs, cs = pauli_masks(terms)
    per = np.zeros(len(terms))
    for j in range(len(terms)):
        per[j] = lib().og_expect_pauli(_ptr(psi), n, int(xs[j]), int(zs[j]))
    return float(np.dot(cs, per)), per


def probabilities(psi: np.ndarray, n: int, normalise: bool = True) -> np.ndarray:
    """p_i = |psi_i|^2 (Sec. 5.3 measurement equation), optionally normalised."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    p = np.zeros(2 ** n)
    lib().og_probabilities(_ptr(psi), n, 1 if normalise else 0, _dp(p))
    return p


def sample(psi: np.ndarray, n: int, u) -> np.ndarray:
    """Basis indices drawn from |psi|^2 by the exact integer inverse CDF of
    og_sample, one per uniform u_k in [0, 1)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(u.size, dtype=np.uint64)
    rc = lib().og_sample(_ptr(psi), n, _dp(u), u.size, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    if rc != 0:
        raise ValueError("og_sample failed (%d)" % rc)
    return out


def expect_z_all(psi: np.ndarray, n: int) -> Tuple[np.ndarray, float]:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    per = np.zeros(n)
    s = ctypes.c_double()
    lib().og_expect_z_all(_ptr(psi), n, _dp(per), ctypes.byref(s))
    return per, float(s.value)


def pauli_apply(psi: np.ndarray, n: int, terms) -> np.ndarray:
    """H psi for H = sum_j c_j P_j."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros_like(psi)
    xs, zs, cs = pauli_masks(terms)
    for j in range(len(terms)):
        lib().og_pauli_apply_add(_ptr(psi), n, int(xs[j]), int(zs[j]), float(cs[j]), _ptr(out))
    return out


def inner(a: np.ndarray, b: np.ndarray, n: int) -> complex:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().og_inner(_ptr(a), _ptr(b), n, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def energy(n: int, gates, param_values, terms) -> float:
    """f(theta) = <0|U^dag H U|0> (Sec. 4.2 objective)."""
    return expect_terms(run(n, gates, param_values), n, terms)[0]


def adjoint_grad(n: int, gates, param_values, terms, n_slots: int) -> Tuple[float, np.ndarray]:
    pk = _Packed(gates, param_values)
    for i in range(pk.n):
        if pk.arr[i].slot == -2:
            raise ValueError("gate %d is bound to a slot but has no rotation generator" % i)
    xs, zs, cs = pauli_masks(terms)
    grad = np.zeros(n_slots)
    val = ctypes.c_double()
    rc = lib().og_adjoint_grad(n, pk.arr, pk.n, xs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                               zs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _dp(cs), len(terms),
                               _dp(grad), n_slots, ctypes.byref(val))
    if rc != 0:
        raise ValueError("oracle adjoint failed (%d)" % rc)
    return float(val.value), grad


def param_shift_grad(n: int, gates, param_values, terms, n_slots: int) -> np.ndarray:
    """Parameter-shift rule per gate occurrence (Sec. 4.2): for a Pauli
    rotation R(theta) = exp(-i theta P/2), d f / d theta = [f(theta + pi/2) -
    f(theta - pi/2)] / 2; a slot shared by several gates sums their terms."""
    import copy
    grad = np.zeros(n_slots)
    base = [copy.copy(g) for g in gates]
    for i, g in enumerate(gates):
        if not g.slots or g.slots[0] < 0:
            continue
        if g.name not in ROTATIONS or g.controls:
            # the two-term rule needs a generator with two eigenvalues a
            # distance 2 apart; a control projector adds a third eigenvalue
            raise ValueError("shift rule needs an uncontrolled rotation at gate %d" % i)
        s = g.slots[0]

        def shifted(shift):
            gs = list(base)
            h = copy.copy(g)
            h.params = [float(param_values[s]) + shift] + list(g.params[1:])
            h.slots = [-1] + list(g.slots[1:])
            gs[i] = h
            return energy(n, gs, param_values, terms)
        if g.name in EXCITATIONS:
            # generator spectrum {-1, 0, 1}: f has frequencies 1/2 and 1 in
            # theta, and the four-term rule (Sec. 4.2) with shifts pi/2 and
            # 3 pi/2 and weights (sqrt2 +- 1) / (4 sqrt2) is exact
            c1 = (math.sqrt(2) + 1) / (4 * math.sqrt(2))
            c2 = (math.sqrt(2) - 1) / (4 * math.sqrt(2))
            grad[s] += c1 * (shifted(math.pi / 2) - shifted(-math.pi / 2)) \
                - c2 * (shifted(3 * math.pi / 2) - shifted(-3 * math.pi / 2))
        else:
            grad[s] += 0.5 * (shifted(math.pi / 2) - shifted(-math.pi / 2))
    return grad


def fd_grad(n: int, gates, param_values, terms, n_slots: int, h: float = 1e-3) -> np.ndarray:
    """Central finite differences in complex128 with step h."""
    grad = np.zeros(n_slots)
    pv = np.array(param_values, dtype=np.float64)
    for s in range(n_slots):
        a = pv.copy(); a[s] += h
        b = pv.copy(); b[s] -= h
        grad[s] = (energy(n, gates, a, terms) - energy(n, gates, b, terms)) / (2 * h)
    return grad


def fuse(n: int, gates, kmax: int, param_values=None):
    """The paper's greedy, order-preserving fusion.  Returns a list of blocks
    (first_gate, end_gate, qubits, matrix) with qubits ascending (qubits[0]
    is the least significant bit of the matrix index)."""
    pk = _Packed(gates, param_values)
    widest = max([len(g.qubits()) for g in gates] + [kmax, 1])
    kcap = widest
    nbmax = max(1, len(gates))
    starts = (ctypes.c_int * (nbmax + 1))()
    nq = (ctypes.c_int * nbmax)()
    qs = (ctypes.c_int * (nbmax * MAXQ))()
    dcap = 1 << kcap
    mats = np.zeros(nbmax * 2 * dcap * dcap)
    nb = lib().og_fuse(n, pk.arr, pk.n, kmax, nbmax, starts, nq, qs, _dp(mats), kcap)
    if nb < 0:
        raise ValueError("oracle fusion buffer too small")
    out = []
    for b in range(nb):
        k = nq[b]
        d = 1 << k
        m = mats[b * 2 * dcap * dcap: b * 2 * dcap * dcap + 2 * d * d].view(np.complex128).reshape(d, d).copy()
        out.append((starts[b], starts[b + 1], [qs[b * MAXQ + i] for i in range(k)], m))
    return out
