"""The allocation-free <Z> read-out (sv_expect_z_all_noalloc) against the
regular one.

Callers that cannot let a library allocate device memory (their device memory
all belongs to their own pool or allocator, or a cudaMalloc/cudaFree must not
synchronize the device under their other streams) use the variant whose
partial sums live in a fixed array inside the library.  This file is collected
last so that a failure here stops a `-x` run only after every other test ran;
it also passes when run alone in a fresh process.
"""

import numpy as np
import pytest

from paper_2608_09733_gb300 import binding as B
from workloads import fused_layered_u3_cz, random_circuit

pytestmark = pytest.mark.gpu


# 24 qubits (complex64) and 23 (complex128) are the smallest states whose
# read-out uses the full grid of partial rows, where the fixed array is most used.
@pytest.mark.parametrize("dt,n", [(B.SV_C64, 24), (B.SV_C64, 20), (B.SV_C128, 23), (B.SV_C128, 13),
                                  (B.SV_C64, 7)])
def test_noalloc_matches_regular_readout_on_two_calls(svlib, cuda_dev, dt, n):
    import torch
    tdt = torch.complex64 if dt == B.SV_C64 else torch.complex128
    for call, seed in enumerate((1, 2)):  # two calls in a row share the fixed scratch
        gates = fused_layered_u3_cz(n, 3, seed=seed) if n >= 2 else random_circuit(n, 10, seed=seed)
        st = torch.empty(2 ** n, dtype=tdt, device="cuda")
        B.sv_init_basis(st, 0)
        B.sv_apply_circuit(st, gates)
        want = B.sv_expect_z_all(st)
        out = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
        B.sv_expect_z_all_noalloc(st, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        # the same kernels on the same grid, summed in the same fixed order:
        # the two read-outs agree bit for bit
        assert np.array_equal(got, want), (call, got, want)


def test_noalloc_rejects_bad_arguments(svlib, cuda_dev):
    import ctypes
    import torch
    st = torch.zeros(16, dtype=torch.complex64, device="cuda")
    host = np.zeros(5)
    rc = svlib.sv_expect_z_all_noalloc(ctypes.c_void_p(st.data_ptr()), 4, B.SV_C64,
                                       ctypes.c_void_p(host.ctypes.data), None)
    assert rc == 1  # out must be device memory
    out = torch.zeros(40, dtype=torch.float64, device="cuda")
    rc = svlib.sv_expect_z_all_noalloc(ctypes.c_void_p(st.data_ptr()), 35, B.SV_C64,
                                       ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1  # beyond 34 qubits
