"""GPU checks of the host copies of states (sv_run_host's state_in and
state_out, sv_set_state, sv_get_state) on both routes: a kernel of SM loads
and stores for page-locked host memory mapped into the device, and
cudaMemcpyAsync for pageable memory and ranges that are not 16-byte aligned
(every state of n >= 1 qubits is a whole number of 16-byte vectors).

Both routes move the same bytes, so every result agrees bit for bit across
them; a circuit with no gates hands the input state back unchanged (an exact
round trip, whatever the route), and the oracle bounds the rest.
"""

import numpy as np
import pytest

import oracle
from paper_2608_09733_gb300 import binding as B
from workloads import fused_layered_u3_cz

pytestmark = pytest.mark.gpu

NP = {B.SV_C64: np.complex64, B.SV_C128: np.complex128}
TOL_STATE = {B.SV_C64: 1e-5, B.SV_C128: 1e-12}


def host_buffers(n, dt, kind):
    """A host array of 2^n amplitudes: 'pageable' (numpy), 'pinned' (a
    page-locked torch tensor, 16-byte aligned) or 'pinned_offset' (the same
    memory one complex64 amplitude in, so 8 bytes off alignment); with the
    object that keeps the memory alive."""
    import torch
    tdt = torch.complex64 if dt == B.SV_C64 else torch.complex128
    if kind == "pageable":
        a = np.zeros(2 ** n, dtype=NP[dt])
        return a, a
    if kind == "pinned":
        t = torch.zeros(2 ** n, dtype=tdt).pin_memory()
        return t.numpy(), t
    t = torch.zeros(2 ** n * (1 if dt == B.SV_C64 else 2) + 1, dtype=torch.complex64).pin_memory()
    raw = t.numpy().view(np.uint8)[8:8 + 2 ** n * np.dtype(NP[dt]).itemsize]
    return raw.view(NP[dt]), t


def random_state(n, dt, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    return (v / np.linalg.norm(v)).astype(NP[dt])


def families(fn):
    B.sv_profile_enable(True)
    try:
        fn()
    finally:
        fam = B.sv_profile_read()
        B.sv_profile_enable(False)
    return fam


@pytest.mark.parametrize("dt", [B.SV_C64, B.SV_C128])
@pytest.mark.parametrize("n", [1, 2, 7, 16])
def test_run_host_routes_agree(svlib, cuda_dev, dt, n):
    gates = fused_layered_u3_cz(n, 3, seed=80 + n)
    init = random_state(n, dt, 5 + n)
    ref = oracle.run(n, gates, init=init.astype(np.complex128))
    outs, zs = {}, {}
    for kind in ("pageable", "pinned", "pinned_offset"):
        sin, keep_in = host_buffers(n, dt, kind)
        sin[:] = init
        sout, keep_out = host_buffers(n, dt, kind)
        zs[kind] = B.sv_run_host(n, dt, gates, fuse_max_k=5, state_in=sin, state_out=sout)
        outs[kind] = sout.copy()
        del keep_in, keep_out
    for kind in ("pinned", "pinned_offset"):
        assert np.array_equal(outs[kind].view(np.uint8), outs["pageable"].view(np.uint8)), kind
        assert np.array_equal(zs[kind], zs["pageable"]), kind
    assert np.max(np.abs(outs["pinned"].astype(np.complex128) - ref)) < TOL_STATE[dt]


@pytest.mark.parametrize("dt,n", [(B.SV_C64, 22), (B.SV_C128, 21), (B.SV_C64, 1)])
def test_empty_circuit_round_trip_is_exact(svlib, cuda_dev, dt, n):
    """A grid-capped copy kernel (2^22 complex64 amplitudes are 2^21 vectors,
    more than one step of the grid) and a one-vector state: with no gates the
    state comes back as it went in, bit for bit, and <Z_q> is the input's."""
    init = random_state(n, dt, 77)
    sin, keep_in = host_buffers(n, dt, "pinned")
    sin[:] = init
    sout, keep_out = host_buffers(n, dt, "pinned")
    sout[:] = 0
    fam = families(lambda: B.sv_run_host(n, dt, [], state_in=sin, state_out=sout))
    assert np.array_equal(sout.view(np.uint8), init.view(np.uint8))
    assert fam["host_load"]["launches"] == 1 and fam["host_store"]["launches"] == 1, fam
    z = B.sv_run_host(n, dt, [], state_in=sin)
    per, _ = oracle.expect_z_all(init.astype(np.complex128), n)
    assert np.max(np.abs(z[:n] - per)) < (1e-5 if dt == B.SV_C64 else 1e-12)


def test_routes_chosen_by_host_memory(svlib, cuda_dev):
    """Mapped page-locked, aligned host memory runs the copy kernels; pageable
    memory and a range 8 bytes off alignment do not."""
    n, dt = 10, B.SV_C64
    init = random_state(n, dt, 3)
    for kind, expect in (("pinned", True), ("pageable", False), ("pinned_offset", False)):
        sin, k1 = host_buffers(n, dt, kind)
        sin[:] = init
        sout, k2 = host_buffers(n, dt, kind)
        fam = families(lambda: B.sv_run_host(n, dt, [], state_in=sin, state_out=sout))
        assert ("host_store" in fam and "host_load" in fam) == expect, (kind, fam)
        assert np.array_equal(sout, init)


def test_library_owned_state_routes(svlib, cuda_dev):
    n = 13
    for dt in (B.SV_C64, B.SV_C128):
        init = random_state(n, dt, 11)
        for kind in ("pinned", "pinned_offset", "pageable"):
            h = B.SvState(n, dt)
            try:
                sin, k1 = host_buffers(n, dt, kind)
                sin[:] = init
                h.set(sin)
                got = h.get()
                assert np.array_equal(got, init), (dt, kind)
                dst, k2 = host_buffers(n, dt, kind)
                B._check(B.load().sv_get_state(h.handle, B.ctypes.c_void_p(dst.ctypes.data), 0))
                assert np.array_equal(dst, init), (dt, kind)
            finally:
                h.free()
