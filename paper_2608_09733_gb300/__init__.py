"""GB300-native state-vector hot path (sm_103a CUDA behind a C ABI).

The package holds the CUDA kernels and host runtime (``csrc/``, built into
``_build/libsv.so`` by ``build.py``), the ctypes binding with the ABI's names
(``binding``), the torch autograd wrapper of the adjoint gradient and the
serving loop.
"""

from .binding import (  # noqa: F401
    SV_C64,
    SV_C128,
    Gates,
    SvError,
    SvState,
    load,
    pauli_terms,
    sv_adjoint_grad,
    sv_adjoint_grad_device,
    sv_adjoint_grad_ex,
    sv_adjoint_grad_rows,
    sv_batch_expect_z,
    sv_batch_expect_z_device,
    sv_apply_circuit,
    sv_apply_circuit_ex,
    SV_BLOCK_AUTO,
    SV_BLOCK_DENSE,
    sv_expect,
    sv_emulate_apply,
    sv_expect_z_all,
    sv_init_basis,
    sv_plan_info,
    sv_probabilities,
    sv_profile_enable,
    sv_profile_read,
    sv_release_scratch,
    sv_jit_set_mode,
    sv_jit_info,
    sv_jit_check,
    sv_jit_check_adjoint,
    sv_run_host,
    sv_run_batch_small,
    sv_sample,
    GateArray,
    layered_u3_cnot_gates,
    sv_version,
)

from .autograd import AdjointExpectation, BatchLayer, adjoint_expectation  # noqa: E402,F401
