"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only *draws* inputs: gate lists (gate name, target and control
qubits, control states, angles, parameter slots), explicit random unitaries
where a workload calls for Haar-random matrices, Pauli Hamiltonians as
(letters, qubits, coefficient) terms, and arrival streams.  It holds none of the
simulator's arithmetic: it never builds a gate matrix from an angle, never
applies a gate and never evaluates an expectation.  The oracle and the CUDA
library each lower these records on their own.

Conventions (Sec. 4.2 and Sec. 9.1 of the paper): qubit q is bit q of the basis
index (little-endian); rotations are R_P(theta) = exp(-i theta P / 2); a gate
names its target(s) before its controls; a control fires on |1> unless its
control state says 0.
"""

from .circuits import (  # noqa: F401
    Gate,
    Term,
    layered_ry_rz_cnot,
    fused_layered_u3_cz,
    precision_sweep,
    hea_ring,
    hea_hamiltonian,
    hea_params,
    serving_stream,
    serving_circuit,
    serving_angles,
    random_circuit,
    random_pauli_terms,
    haar_unitary,
    haar_u3_angles,
    ghz_circuit,
    qft_circuit,
)
