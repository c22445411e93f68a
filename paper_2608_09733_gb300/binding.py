"""ctypes binding of libsv.so: argument marshalling only.

Every function here has the name of the C entry point it calls (see
include/sv.h) and does nothing but convert Python arguments (gate records,
Pauli terms, torch tensors, the current torch stream) into the C structs and
pointers of the ABI, call it, and raise ``SvError`` on a non-OK status.  All
arithmetic runs in the library's CUDA kernels; there is no CPU path.  When
libsv.so has not been built, loading fails with an error that says how to
build it.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsv.so")

SV_C64, SV_C128 = 0, 1
STATUS = {0: "SV_OK", 1: "SV_ERR_INVALID", 2: "SV_ERR_UNSUPPORTED", 3: "SV_ERR_OOM", 4: "SV_ERR_CUDA",
          5: "SV_ERR_TIMEOUT", 6: "SV_ERR_UNBOUND_PARAM"}
SV_ERR_INVALID = 1

GATE_TYPES = {
    "i": 0, "x": 1, "y": 2, "z": 3, "h": 4, "s": 5, "sdg": 6, "t": 7, "tdg": 8, "sx": 9,
    "rx": 10, "ry": 11, "rz": 12, "p": 13, "u2": 14, "u3": 15,
    "swap": 16, "rxx": 17, "ryy": 18, "rzz": 19, "unitary": 20,
    "exc1": 21, "exc2": 22,
}

# Every symbol include/sv.h declares (checked by the CPU tests).
EXPORTS = ["sv_version", "sv_last_error", "sv_init_basis", "sv_apply_circuit", "sv_apply_circuit_ex", "sv_expect",
           "sv_expect_z_all",
           "sv_plan_info", "sv_run_host", "sv_alloc", "sv_free", "sv_state_ptr", "sv_set_state", "sv_get_state",
           "sv_release_scratch", "sv_profile_enable", "sv_profile_read", "sv_adjoint_grad", "sv_run_batch_small",
           "sv_expect_z_all_noalloc", "sv_emulate_apply", "sv_probabilities", "sv_sample", "sv_adjoint_grad_rows",
           "sv_batch_expect_z", "sv_adjoint_grad_ex", "sv_adjoint_grad_device", "sv_batch_expect_z_device",
           "sv_small_session_start", "sv_small_session_submit", "sv_small_session_poll", "sv_small_session_stop",
           "sv_jit_set_mode", "sv_jit_info", "sv_jit_check", "sv_jit_check_adjoint"]


class SvError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS.get(status, str(status)), message))
        self.status = status
        self.name = STATUS.get(status, str(status))


class SvGate(ctypes.Structure):
    _fields_ = [
        ("type", ctypes.c_int32),
        ("n_targets", ctypes.c_int32),
        ("targets", ctypes.c_int32 * 5),
        ("n_controls", ctypes.c_int32),
        ("controls", ctypes.c_int32 * 5),
        ("control_zero_mask", ctypes.c_uint32),
        ("param_slot", ctypes.c_int32 * 3),
        ("params", ctypes.c_double * 3),
        ("matrix", ctypes.POINTER(ctypes.c_double)),
    ]


class SvExecOpts(ctypes.Structure):
    _fields_ = [("fuse_max_k", ctypes.c_int32), ("block_mode", ctypes.c_int32), ("ops_per_pass", ctypes.c_int32),
                ("tile_qubits", ctypes.c_int32)]


SV_BLOCK_AUTO, SV_BLOCK_DENSE = 0, 1


class SvProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class SvAdjointOpts(ctypes.Structure):
    _fields_ = [("checkpoint_every", ctypes.c_int32), ("stored_states", ctypes.c_int32),
                ("memory_budget_bytes", ctypes.c_double)]


class SvPauliTerm(ctypes.Structure):
    _fields_ = [("x_mask", ctypes.c_uint64), ("z_mask", ctypes.c_uint64), ("coeff", ctypes.c_double)]


_lib = None


def load():
    """Loads libsv.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsv.so is not built (%s); run `python -m paper_2608_09733_gb300.build` "
                               "or __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, vp, sz, cd = ctypes.POINTER, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_double
        ci = ctypes.c_int
        sig = {
            "sv_version": ([], ci),
            "sv_last_error": ([], ctypes.c_char_p),
            "sv_init_basis": ([vp, ci, ci, ctypes.c_uint64, vp], ci),
            "sv_apply_circuit": ([vp, ci, ci, P(SvGate), sz, P(cd), sz, ci, vp], ci),
            "sv_expect": ([vp, ci, ci, P(SvPauliTerm), sz, vp, ci, vp], ci),
            "sv_expect_z_all": ([vp, ci, ci, vp, ci, vp], ci),
            "sv_apply_circuit_ex": ([vp, ci, ci, P(SvGate), sz, P(cd), sz, P(SvExecOpts), vp], ci),
            "sv_plan_info": ([ci, ci, P(SvGate), sz, P(cd), sz, P(SvExecOpts), P(ci), P(ci), P(ci)], ci),
            "sv_emulate_apply": ([ci, ci, P(SvGate), sz, P(cd), sz, P(SvExecOpts), vp], ci),
            "sv_probabilities": ([vp, ci, ci, vp, ci, vp], ci),
            "sv_sample": ([vp, ci, ci, P(cd), sz, vp, ci, vp], ci),
            "sv_adjoint_grad_rows": ([ci, ci, P(SvGate), sz, P(cd), ci, ci, P(SvPauliTerm), sz, P(cd), ci, P(cd),
                                      P(cd), vp], ci),
            "sv_batch_expect_z": ([ci, ci, P(SvGate), sz, P(cd), ci, ci, P(cd), vp], ci),
            "sv_adjoint_grad_ex": ([ci, ci, P(SvGate), sz, P(cd), ci, ci, P(SvPauliTerm), sz, P(SvAdjointOpts),
                                    P(cd), P(cd), vp], ci),
            "sv_run_host": ([ci, ci, vp, P(SvGate), sz, P(cd), sz, ci, P(cd), vp, vp], ci),
            "sv_alloc": ([ci, ci, vp, P(vp)], ci),
            "sv_free": ([vp], ci),
            "sv_state_ptr": ([vp], vp),
            "sv_set_state": ([vp, vp, ci], ci),
            "sv_get_state": ([vp, vp, ci], ci),
            "sv_release_scratch": ([], ci),
            "sv_profile_enable": ([ci], ci),
            "sv_adjoint_grad": ([ci, ci, P(SvGate), sz, P(cd), ci, ci, P(SvPauliTerm), sz, ci, P(cd), P(cd), vp], ci),
            "sv_run_batch_small": ([ci, ci, P(ci), P(P(SvGate)), P(sz), vp, ci, vp], ci),
            "sv_expect_z_all_noalloc": ([vp, ci, ci, vp, vp], ci),
            "sv_profile_read": ([P(SvProfileEntry), ci, P(ci), ci], ci),
            "sv_adjoint_grad_device": ([ci, ci, P(SvGate), sz, vp, ci, ci, P(SvPauliTerm), sz, vp, ci, vp, vp, vp],
                                       ci),
            "sv_batch_expect_z_device": ([ci, ci, P(SvGate), sz, vp, ci, ci, vp, vp], ci),
            "sv_small_session_start": ([ci, ci, ci, cd, ci, P(vp)], ci),
            "sv_small_session_submit": ([vp, ci, P(ci), P(P(SvGate)), P(sz), P(ctypes.c_int64)], ci),
            "sv_small_session_poll": ([vp, ctypes.c_int64, P(cd), P(ci)], ci),
            "sv_small_session_stop": ([vp], ci),
            "sv_jit_set_mode": ([ci], ci),
            "sv_jit_info": ([P(ci), P(ci), P(ctypes.c_longlong), P(ctypes.c_longlong), P(ctypes.c_longlong), P(cd),
                             ctypes.c_char_p, sz], ci),
            "sv_jit_check": ([ci, ci, P(SvGate), sz, P(cd), sz, P(SvExecOpts), ci, ci, P(ci), P(ci), ctypes.c_char_p,
                              sz], ci),
            "sv_jit_check_adjoint": ([ci, ci, P(SvGate), sz, ci, ci, ci, ci, P(ci), P(ci), ctypes.c_char_p, sz], ci),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise SvError(status, load().sv_last_error().decode(errors="replace"))


# ---------------------------------------------------------------- marshalling

# numpy view of SvGate with the same field offsets (the matrix pointer as u8)
GATE_DTYPE = np.dtype({
    "names": ["type", "n_targets", "targets", "n_controls", "controls", "control_zero_mask", "param_slot", "params",
              "matrix"],
    "formats": ["<i4", "<i4", ("<i4", 5), "<i4", ("<i4", 5), "<u4", ("<i4", 3), ("<f8", 3), "<u8"],
    "offsets": [getattr(SvGate, f).offset for f in ("type", "n_targets", "targets", "n_controls", "controls",
                                                     "control_zero_mask", "param_slot", "params", "matrix")],
    "itemsize": ctypes.sizeof(SvGate),
})


class GateArray:
    """SvGate records held in a numpy structured array (built without a
    per-gate Python loop); quacks like ``Gates``."""

    def __init__(self, arr: np.ndarray):
        assert arr.dtype == GATE_DTYPE
        self.np = np.ascontiguousarray(arr)
        self.n = len(self.np)
        self.arr = self.np.ctypes.data_as(ctypes.POINTER(SvGate))


def layered_u3_cnot_gates(n: int, angles: np.ndarray) -> GateArray:
    """Gate records of ``depth`` layers of U3(angles[d, q]) on every qubit
    followed by the CNOT ladder q -> q+1 (the serving workload's circuit)."""
    depth = angles.shape[0]
    per = 2 * n - 1
    a = np.zeros(depth * per, dtype=GATE_DTYPE)
    a["param_slot"][:] = -1
    base = (np.arange(depth) * per)[:, None]
    u3 = (base + np.arange(n)[None, :]).ravel()
    a["type"][u3] = GATE_TYPES["u3"]
    a["n_targets"][u3] = 1
    a["targets"][u3, 0] = np.tile(np.arange(n), depth)
    a["params"][u3] = angles.reshape(-1, 3)
    if n > 1:
        cx = (base + n + np.arange(n - 1)[None, :]).ravel()
        a["type"][cx] = GATE_TYPES["x"]
        a["n_targets"][cx] = 1
        a["targets"][cx, 0] = np.tile(np.arange(1, n), depth)
        a["n_controls"][cx] = 1
        a["controls"][cx, 0] = np.tile(np.arange(n - 1), depth)
    return GateArray(a)


class Gates:
    """A ctypes array of SvGate built from gate records (workloads.Gate or any
    object with name/targets/controls/control_states/params/slots/matrix)."""

    def __init__(self, gates):
        self._keep = []
        self.n = len(gates)
        self.arr = (SvGate * max(1, self.n))()
        for i, g in enumerate(gates):
            o = self.arr[i]
            o.type = GATE_TYPES[g.name]
            o.n_targets = len(g.targets)
            o.n_controls = len(g.controls)
            for j, q in enumerate(g.targets):
                o.targets[j] = q
            mask = 0
            for j, q in enumerate(g.controls):
                o.controls[j] = q
                if int(g.control_states[j]) == 0:
                    mask |= 1 << j
            o.control_zero_mask = mask
            slots = list(g.slots) + [-1] * (3 - len(g.slots))
            params = list(g.params) + [0.0] * (3 - len(g.params))
            for j in range(3):
                o.param_slot[j] = int(slots[j])
                o.params[j] = float(params[j])
            if g.name == "unitary":
                buf = np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128)).view(np.float64).reshape(-1)
                buf = np.ascontiguousarray(buf)
                self._keep.append(buf)
                o.matrix = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def pauli_terms(terms) -> "ctypes.Array":
    """ctypes array of SvPauliTerm from (paulis, qubits, coeff) records."""
    arr = (SvPauliTerm * max(1, len(terms)))()
    for j, t in enumerate(terms):
        x = z = 0
        for letter, q in zip(t.paulis, t.qubits):
            if letter in "XY":
                x |= 1 << q
            if letter in "ZY":
                z |= 1 << q
        arr[j].x_mask, arr[j].z_mask, arr[j].coeff = x, z, float(t.coeff)
    return arr


def _params(param_values):
    if param_values is None:
        return None, 0, None
    pv = np.ascontiguousarray(np.asarray(param_values, dtype=np.float64).reshape(-1))
    return pv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pv.size, pv


def _dtype_of(t) -> int:
    import torch
    if t.dtype == torch.complex64:
        return SV_C64
    if t.dtype == torch.complex128:
        return SV_C128
    raise TypeError("state must be complex64 or complex128, got %s" % t.dtype)


def _n_of(t) -> int:
    n = int(t.numel()).bit_length() - 1
    if t.numel() != (1 << n) or not t.is_contiguous():
        raise ValueError("state must be a contiguous tensor of 2^n amplitudes")
    return n


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------- entry points

def sv_version() -> int:
    return int(load().sv_version())


def sv_init_basis(state, basis_index: int = 0, stream=None):
    _check(load().sv_init_basis(ctypes.c_void_p(state.data_ptr()), _n_of(state), _dtype_of(state),
                                int(basis_index), _stream(stream)))


def sv_apply_circuit(state, gates, param_values=None, fuse_max_k: int = 0, stream=None):
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    pp, npv, _keep = _params(param_values)
    _check(load().sv_apply_circuit(ctypes.c_void_p(state.data_ptr()), _n_of(state), _dtype_of(state), g.arr, g.n,
                                   pp, npv, int(fuse_max_k), _stream(stream)))


def _opts(fuse_max_k=0, block_mode=0, ops_per_pass=0, tile_qubits=0):
    o = SvExecOpts()
    o.fuse_max_k, o.block_mode, o.ops_per_pass = int(fuse_max_k), int(block_mode), int(ops_per_pass)
    o.tile_qubits = int(tile_qubits)
    return o


def sv_apply_circuit_ex(state, gates, param_values=None, fuse_max_k: int = 0, block_mode: int = 0,
                        ops_per_pass: int = 0, stream=None, tile_qubits: int = 0):
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    pp, npv, _keep = _params(param_values)
    o = _opts(fuse_max_k, block_mode, ops_per_pass, tile_qubits)
    _check(load().sv_apply_circuit_ex(ctypes.c_void_p(state.data_ptr()), _n_of(state), _dtype_of(state), g.arr, g.n,
                                      pp, npv, ctypes.byref(o), _stream(stream)))


def sv_expect(state, terms, out=None, stream=None) -> np.ndarray:
    """<P_j> per term; into a device float64 tensor `out` if given (async),
    else returned as a host array."""
    arr = terms if isinstance(terms, ctypes.Array) else pauli_terms(terms)
    nt = len(arr) if isinstance(terms, ctypes.Array) else len(terms)
    if out is None:
        host = np.zeros(nt, dtype=np.float64)
        _check(load().sv_expect(ctypes.c_void_p(state.data_ptr()), _n_of(state), _dtype_of(state), arr, nt,
                                host.ctypes.data_as(ctypes.c_void_p), 0, _stream(stream)))
        return host
    _check(load().sv_expect(ctypes.c_void_p(state.data_ptr()), _n_of(state), _dtype_of(state), arr, nt,
                            ctypes.c_void_p(out.data_ptr()), 1, _stream(stream)))
    return out


def sv_expect_z_all(state, out=None, stream=None):
    """(<Z_q> for all q, their sum) as a host array of n + 1, or written into a
    device float64 tensor `out` (async)."""
    n = _n_of(state)
    if out is None:
        host = np.zeros(n + 1, dtype=np.float64)
        _check(load().sv_expect_z_all(ctypes.c_void_p(state.data_ptr()), n, _dtype_of(state),
                                      host.ctypes.data_as(ctypes.c_void_p), 0, _stream(stream)))
        return host
    _check(load().sv_expect_z_all(ctypes.c_void_p(state.data_ptr()), n, _dtype_of(state),
                                  ctypes.c_void_p(out.data_ptr()), 1, _stream(stream)))
    return out


def sv_plan_info(n: int, dtype: int, gates, param_values=None, fuse_max_k: int = 0, block_mode: int = 0,
                 ops_per_pass: int = 0, tile_qubits: int = 0):
    """(number of blocks, number of HBM passes, block start indices)."""
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    pp, npv, _keep = _params(param_values)
    nb, ns = ctypes.c_int(), ctypes.c_int()
    starts = (ctypes.c_int * (g.n + 1))()
    o = _opts(fuse_max_k, block_mode, ops_per_pass, tile_qubits)
    _check(load().sv_plan_info(n, dtype, g.arr, g.n, pp, npv, ctypes.byref(o), ctypes.byref(nb), ctypes.byref(ns),
                               starts))
    return nb.value, ns.value, [starts[i] for i in range(nb.value + 1)]


def sv_probabilities(state, normalise: bool = True, out=None, stream=None):
    """|psi_i|^2 as a device float64 tensor (normalised by default)."""
    import torch
    n = _n_of(state)
    if out is None:
        out = torch.empty(1 << n, dtype=torch.float64, device=state.device)
    _check(load().sv_probabilities(ctypes.c_void_p(state.data_ptr()), n, _dtype_of(state),
                                   ctypes.c_void_p(out.data_ptr()), 1 if normalise else 0, _stream(stream)))
    return out


def sv_sample(state, uniforms, out=None, stream=None) -> np.ndarray:
    """Basis indices drawn from |psi|^2, one per uniform in [0, 1) (host
    numpy array); into the device uint64-compatible tensor ``out`` (int64)
    if given, else returned as a numpy uint64 array."""
    n = _n_of(state)
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    if out is not None:
        _check(load().sv_sample(ctypes.c_void_p(state.data_ptr()), n, _dtype_of(state),
                                u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), u.size,
                                ctypes.c_void_p(out.data_ptr()), 1, _stream(stream)))
        return out
    host = np.zeros(u.size, dtype=np.uint64)
    _check(load().sv_sample(ctypes.c_void_p(state.data_ptr()), n, _dtype_of(state),
                            u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), u.size,
                            ctypes.c_void_p(host.ctypes.data), 0, _stream(stream)))
    return host


def sv_emulate_apply(state: np.ndarray, n: int, dtype: int, gates, param_values=None, fuse_max_k: int = 0,
                     block_mode: int = 0, ops_per_pass: int = 0, tile_qubits: int = 0) -> np.ndarray:
    """Runs the kernel programs the plan of `gates` builds for `dtype` on the
    host, in double precision, on a complex128 numpy state (in place)."""
    assert state.dtype == np.complex128 and state.size == 1 << n and state.flags.c_contiguous
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    pp, npv, _keep = _params(param_values)
    o = _opts(fuse_max_k, block_mode, ops_per_pass, tile_qubits)
    _check(load().sv_emulate_apply(n, dtype, g.arr, g.n, pp, npv, ctypes.byref(o),
                                   ctypes.c_void_p(state.ctypes.data)))
    return state


def _host_state(a, n: int, dtype: int, what: str, writable: bool = False):
    """Pointer to a host array holding exactly 2^n amplitudes of dtype: the C
    side copies that many bytes, so a shorter, strided or read-only target is
    refused here."""
    want = np.complex64 if dtype == SV_C64 else np.complex128
    if not isinstance(a, np.ndarray) or a.dtype != want or a.size != (1 << n) or not a.flags.c_contiguous:
        raise SvError(SV_ERR_INVALID, "%s must be a C-contiguous %s numpy array of 2^%d amplitudes"
                      % (what, np.dtype(want).name, n))
    if writable and not a.flags.writeable:
        raise SvError(SV_ERR_INVALID, "%s is read-only" % what)
    return ctypes.c_void_p(a.ctypes.data)


def sv_run_host(n: int, dtype: int, gates, param_values=None, fuse_max_k: int = 0, state_in=None,
                state_out=None, stream=None) -> np.ndarray:
    """End-to-end on host buffers (numpy): returns (<Z_q>..., sum)."""
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    pp, npv, _keep = _params(param_values)
    out = np.zeros(n + 1, dtype=np.float64)
    sin = _host_state(state_in, n, dtype, "state_in") if state_in is not None else None
    sout = _host_state(state_out, n, dtype, "state_out", writable=True) if state_out is not None else None
    st = _stream(stream) if stream is not None else ctypes.c_void_p(0)
    _check(load().sv_run_host(n, dtype, sin, g.arr, g.n, pp, npv, int(fuse_max_k),
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), sout, st))
    return out


class SvState:
    """A library-owned state (sv_alloc / sv_free)."""

    def __init__(self, n: int, dtype: int, stream=None):
        self.n, self.dtype = n, dtype
        h = ctypes.c_void_p()
        st = _stream(stream) if stream is not None else ctypes.c_void_p(0)
        _check(load().sv_alloc(n, dtype, st, ctypes.byref(h)))
        self.handle = h

    @property
    def ptr(self) -> int:
        return load().sv_state_ptr(self.handle)

    def set(self, host: np.ndarray):
        _check(load().sv_set_state(self.handle, _host_state(host, self.n, self.dtype, "host"), 0))

    def get(self) -> np.ndarray:
        out = np.zeros(1 << self.n, dtype=np.complex64 if self.dtype == SV_C64 else np.complex128)
        _check(load().sv_get_state(self.handle, ctypes.c_void_p(out.ctypes.data), 0))
        return out

    def free(self):
        if self.handle:
            _check(load().sv_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sv_release_scratch():
    _check(load().sv_release_scratch())


def sv_jit_set_mode(mode: int):
    """0: never compile pass programs; 1 (default): compile a program
    structure on its second use (by any circuit of the same gates, at any
    angles); 2: on its first; -1: the SV_JIT environment variable."""
    _check(load().sv_jit_set_mode(int(mode)))


def sv_jit_info() -> dict:
    """Mode, NVRTC availability, kernels compiled / failed, launches of
    compiled kernels, host seconds spent compiling and the last message."""
    mode, av = ctypes.c_int(), ctypes.c_int()
    comp, fail, launches = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    secs = ctypes.c_double()
    msg = ctypes.create_string_buffer(4096)
    _check(load().sv_jit_info(ctypes.byref(mode), ctypes.byref(av), ctypes.byref(comp), ctypes.byref(fail),
                              ctypes.byref(launches), ctypes.byref(secs), msg, 4096))
    return {"mode": mode.value, "available": bool(av.value), "compiled": comp.value, "failed": fail.value,
            "launches": launches.value, "compile_seconds": secs.value, "message": msg.value.decode(errors="replace")}


def sv_jit_check(n: int, dtype: int, gates, param_values=None, fuse_max_k: int = 0, compile: bool = True,
                 arch: int = 103, block_mode: int = 0, ops_per_pass: int = 0, tile_qubits: int = 0):
    """(sources, compiled, text): the passes of a circuit that would run as
    compiled kernels, how many compiled for sm_<arch>a (no device needed),
    and the first compile error or else every source (each followed by a
    "// ----" line)."""
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    pp, npv, _keep = _params(param_values)
    o = _opts(fuse_max_k, block_mode, ops_per_pass, tile_qubits)
    ns, nc = ctypes.c_int(), ctypes.c_int()
    cap = 1 << 23
    buf = ctypes.create_string_buffer(cap)
    _check(load().sv_jit_check(n, dtype, g.arr, g.n, pp, npv, ctypes.byref(o), 1 if compile else 0, arch,
                               ctypes.byref(ns), ctypes.byref(nc), buf, cap))
    return ns.value, nc.value, buf.value.decode(errors="replace")


def sv_jit_check_adjoint(n: int, dtype: int, gates, n_params: int, checkpoint_every: int = 0, compile: bool = True,
                         arch: int = 103):
    """(sources, compiled, text) for the batched forward and reverse passes of
    an adjoint template: the distinct kernels written, how many compiled for
    sm_<arch>a (no device needed), and the first compile error or else every
    source."""
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    ns, nc = ctypes.c_int(), ctypes.c_int()
    cap = 1 << 23
    buf = ctypes.create_string_buffer(cap)
    _check(load().sv_jit_check_adjoint(n, dtype, g.arr, g.n, int(n_params), int(checkpoint_every),
                                       1 if compile else 0, arch, ctypes.byref(ns), ctypes.byref(nc), buf, cap))
    return ns.value, nc.value, buf.value.decode(errors="replace")


def sv_profile_enable(on: bool = True):
    _check(load().sv_profile_enable(1 if on else 0))


def sv_profile_read(reset: bool = True) -> dict:
    """{family: {"launches", "total_ms", "bytes"}} of the launches recorded
    since profiling was enabled (waits for their events)."""
    arr = (SvProfileEntry * 64)()
    n = ctypes.c_int()
    _check(load().sv_profile_read(arr, 64, ctypes.byref(n), 1 if reset else 0))
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "total_ms": float(arr[i].total_ms),
                                   "bytes": float(arr[i].bytes)} for i in range(min(n.value, 64))}


def sv_adjoint_grad(n: int, dtype: int, gates, params, terms, checkpoint_every: int = 0, stream=None):
    """(values (batch,), gradients (batch, n_params)) for a (batch, n_params)
    array of parameter vectors (host float64)."""
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    pv = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    if pv.ndim == 1:
        pv = pv.reshape(1, -1)
    batch, npar = pv.shape
    arr = terms if isinstance(terms, ctypes.Array) else pauli_terms(terms)
    nt = len(arr)
    grad = np.zeros((batch, npar), dtype=np.float64)
    val = np.zeros(batch, dtype=np.float64)
    st = _stream(stream) if stream is not None else ctypes.c_void_p(0)
    _check(load().sv_adjoint_grad(n, dtype, g.arr, g.n, pv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), batch,
                                  npar, arr, nt, int(checkpoint_every),
                                  grad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  val.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), st))
    return val, grad


def sv_adjoint_grad_ex(n: int, dtype: int, gates, params, terms, checkpoint_every: int = 0,
                       stored_states: int = -1, memory_budget_bytes: float = 0.0, stream=None):
    """sv_adjoint_grad with a checkpoint policy: keep stored_states of the
    segment-start states (-1: all) or as many as memory_budget_bytes holds;
    the others are recomputed in the reverse pass."""
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    pv = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    if pv.ndim == 1:
        pv = pv.reshape(1, -1)
    batch, npar = pv.shape
    arr = terms if isinstance(terms, ctypes.Array) else pauli_terms(terms)
    grad = np.zeros((batch, npar), dtype=np.float64)
    val = np.zeros(batch, dtype=np.float64)
    o = SvAdjointOpts(int(checkpoint_every), int(stored_states), float(memory_budget_bytes))
    st = _stream(stream) if stream is not None else ctypes.c_void_p(0)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().sv_adjoint_grad_ex(n, dtype, g.arr, g.n, pv.ctypes.data_as(dp), batch, npar, arr, len(arr),
                                     ctypes.byref(o), grad.ctypes.data_as(dp), val.ctypes.data_as(dp), st))
    return val, grad


def sv_adjoint_grad_rows(n: int, dtype: int, gates, params, terms, row_coeffs, checkpoint_every: int = 0,
                         stream=None):
    """sv_adjoint_grad with H_b = sum_j row_coeffs[b, j] P_j per state:
    (values (batch,), gradients (batch, n_params))."""
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    pv = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    if pv.ndim == 1:
        pv = pv.reshape(1, -1)
    batch, npar = pv.shape
    arr = terms if isinstance(terms, ctypes.Array) else pauli_terms(terms)
    nt = len(arr)
    rc = np.ascontiguousarray(np.asarray(row_coeffs, dtype=np.float64))
    if rc.shape != (batch, nt):
        raise ValueError("row_coeffs must be (batch, n_terms) = (%d, %d)" % (batch, nt))
    grad = np.zeros((batch, npar), dtype=np.float64)
    val = np.zeros(batch, dtype=np.float64)
    st = _stream(stream) if stream is not None else ctypes.c_void_p(0)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().sv_adjoint_grad_rows(n, dtype, g.arr, g.n, pv.ctypes.data_as(dp), batch, npar, arr, nt,
                                       rc.ctypes.data_as(dp), int(checkpoint_every), grad.ctypes.data_as(dp),
                                       val.ctypes.data_as(dp), st))
    return val, grad


def sv_batch_expect_z(n: int, dtype: int, gates, params, stream=None) -> np.ndarray:
    """(batch, n + 1): <Z_q> of U(params_b)|0..0> for every qubit, then their sum."""
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    pv = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    if pv.ndim == 1:
        pv = pv.reshape(1, -1)
    batch, npar = pv.shape
    out = np.zeros((batch, n + 1), dtype=np.float64)
    st = _stream(stream) if stream is not None else ctypes.c_void_p(0)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().sv_batch_expect_z(n, dtype, g.arr, g.n, pv.ctypes.data_as(dp), batch, npar, out.ctypes.data_as(dp),
                                    st))
    return out


def _dev_ptr(t, what):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("%s must be a contiguous float64 CUDA tensor" % what)
    return ctypes.c_void_p(t.data_ptr())


def sv_adjoint_grad_device(n: int, dtype: int, gates, params, terms, row_coeffs=None, checkpoint_every: int = 0,
                           out_grad=None, out_value=None, values_only: bool = False, stream=None):
    """Device-array adjoint (nothing is copied to the host; asynchronous on
    `stream`).  params: (batch, n_params) float64 CUDA tensor; row_coeffs:
    (batch, n_terms) CUDA tensor or None.  Returns (values, gradients) as CUDA
    tensors; gradients is None when values_only."""
    import torch
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    p = params if params.dim() == 2 else params.reshape(1, -1)
    batch, npar = p.shape
    arr = terms if isinstance(terms, ctypes.Array) else pauli_terms(terms)
    if out_value is None:
        out_value = torch.empty(batch, dtype=torch.float64, device=p.device)
    if out_grad is None and not values_only:
        out_grad = torch.empty((batch, npar), dtype=torch.float64, device=p.device)
    rc = _dev_ptr(row_coeffs, "row_coeffs") if row_coeffs is not None else ctypes.c_void_p(0)
    og = _dev_ptr(out_grad, "out_grad") if not values_only else ctypes.c_void_p(0)
    st = _stream(stream) if stream is not None else _stream(torch.cuda.current_stream())
    _check(load().sv_adjoint_grad_device(n, dtype, g.arr, g.n, _dev_ptr(p, "params"), batch, npar, arr, len(arr), rc,
                                         int(checkpoint_every), og, _dev_ptr(out_value, "out_value"), st))
    return out_value, (None if values_only else out_grad)


def sv_batch_expect_z_device(n: int, dtype: int, gates, params, out=None, stream=None):
    """(batch, n + 1) CUDA tensor: <Z_q> of U(params_b)|0..0> per qubit, then
    their sum; params a (batch, n_params) float64 CUDA tensor (asynchronous)."""
    import torch
    g = gates if isinstance(gates, (Gates, GateArray)) else Gates(gates)
    p = params if params.dim() == 2 else params.reshape(1, -1)
    batch, npar = p.shape
    if out is None:
        out = torch.empty((batch, n + 1), dtype=torch.float64, device=p.device)
    st = _stream(stream) if stream is not None else _stream(torch.cuda.current_stream())
    _check(load().sv_batch_expect_z_device(n, dtype, g.arr, g.n, _dev_ptr(p, "params"), batch, npar,
                                           _dev_ptr(out, "out"), st))
    return out


SV_SESSION_MAX_QUBITS = 14


class SmallSession:
    """A resident packed kernel fed from a work queue (sv_small_session_*):
    submit small requests (n <= 14 complex64, 12 complex128), poll tickets,
    stop.  ``stop`` raises SvError(SV_ERR_TIMEOUT) when a device-side wait of
    the session ran out (it sat idle past ``wait_limit_s``)."""

    def __init__(self, dtype: int = SV_C64, capacity: int = 16384, arena_programs: int = 8192,
                 wait_limit_s: float = 0.05, n_ctas: int = 0):
        self.h = ctypes.c_void_p()
        self.dtype = dtype
        _check(load().sv_small_session_start(dtype, capacity, arena_programs, float(wait_limit_s), n_ctas,
                                             ctypes.byref(self.h)))

    def submit(self, n_qubits, gate_sets):
        """Plans and publishes the requests; returns their tickets."""
        nreq = len(gate_sets)
        gs = [g if isinstance(g, (Gates, GateArray)) else Gates(g) for g in gate_sets]
        nq = (ctypes.c_int * nreq)(*[int(v) for v in n_qubits])
        ptrs = (ctypes.POINTER(SvGate) * nreq)(*[g.arr for g in gs])
        ngs = (ctypes.c_size_t * nreq)(*[g.n for g in gs])
        tk = (ctypes.c_int64 * nreq)()
        _check(load().sv_small_session_submit(self.h, nreq, nq, ptrs, ngs, tk))
        return [int(t) for t in tk]

    def poll(self, ticket: int):
        """(done, sum_q <Z_q>) of a ticket; never waits."""
        r, d = ctypes.c_double(), ctypes.c_int()
        _check(load().sv_small_session_poll(self.h, int(ticket), ctypes.byref(r), ctypes.byref(d)))
        return bool(d.value), float(r.value)

    def stop(self):
        if self.h:
            h, self.h = self.h, ctypes.c_void_p()
            _check(load().sv_small_session_stop(h))


def sv_run_batch_small(n_qubits, gate_sets, dtype: int = SV_C64, out=None, stream=None):
    """Packed launch of small requests: gate_sets[b] (Gates/GateArray or a
    gate list) on n_qubits[b] qubits; returns sum_q <Z_q> per request (host),
    or writes them into the device float64 tensor ``out`` (async)."""
    nreq = len(gate_sets)
    gs = [g if isinstance(g, (Gates, GateArray)) else Gates(g) for g in gate_sets]
    nq = (ctypes.c_int * nreq)(*[int(x) for x in n_qubits])
    ptrs = (ctypes.POINTER(SvGate) * nreq)(*[ctypes.cast(g.arr, ctypes.POINTER(SvGate)) for g in gs])
    ng = (ctypes.c_size_t * nreq)(*[g.n for g in gs])
    st = _stream(stream) if stream is not None else ctypes.c_void_p(0)
    if out is None:
        host = np.zeros(nreq, dtype=np.float64)
        _check(load().sv_run_batch_small(nreq, dtype, nq, ptrs, ng, host.ctypes.data_as(ctypes.c_void_p), 0, st))
        return host
    _check(load().sv_run_batch_small(nreq, dtype, nq, ptrs, ng, ctypes.c_void_p(out.data_ptr()), 1, st))
    return out


def sv_expect_z_all_noalloc(state, out, stream=None):
    """sv_expect_z_all into the device float64 tensor ``out`` (n + 1) with the
    library's fixed scratch array instead of allocated scratch (async)."""
    _check(load().sv_expect_z_all_noalloc(ctypes.c_void_p(state.data_ptr()), _n_of(state), _dtype_of(state),
                                          ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out
