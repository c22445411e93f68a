"""The pass-kernel generator and the run-time compiler, without a GPU.

sv_jit_check plans a circuit, writes the kernel source of every pass the TMA
pass would run and compiles each with NVRTC for sm_103a; no device is
touched.  Results of the compiled kernels are checked on the GPU
(test_gpu_jit.py).
"""

import re

import pytest

from paper_2608_09733_gb300 import binding as B
from workloads import fused_layered_u3_cz, random_circuit


def _nvrtc_or_skip():
    info = B.sv_jit_info()
    if not info["available"]:
        pytest.skip("NVRTC not available: " + info["message"])


def test_sources_only_for_tma_passes(svlib):
    g = fused_layered_u3_cz(20, 4, seed=1)
    # 20 qubits with 12-qubit tiles: 2^8 tiles, fewer than the TMA pass takes
    assert B.sv_jit_check(20, B.SV_C64, g, fuse_max_k=5, compile=False)[0] == 0
    # complex128 passes are not compiled
    g = fused_layered_u3_cz(26, 4, seed=1)
    assert B.sv_jit_check(26, B.SV_C128, g, fuse_max_k=5, compile=False)[0] == 0
    _, passes, _ = B.sv_plan_info(26, B.SV_C64, g, fuse_max_k=5)
    ns, nc, src = B.sv_jit_check(26, B.SV_C64, g, fuse_max_k=5, compile=False)
    assert ns == passes and nc == 0
    assert "k_sweep_jit" in src and "tma_pass_body" in src


def test_generated_source_has_constant_dispatch(svlib):
    """The layered U3/CZ circuit's passes are phase tables, rotations and sign
    flips only: no op descriptor is read at run time in a register phase."""
    g = fused_layered_u3_cz(26, 6, seed=2)
    _, _, src = B.sv_jit_check(26, B.SV_C64, g, fuse_max_k=5, compile=False)
    assert "r_rot<float, 5," in src and "r_phase_table<float, 5>" in src
    assert "P.ops[" not in src
    # every register phase stages its 32 amplitudes: m[] holds five distinct bits
    for ms in re.findall(r"const uint32_t m\[5\] = \{([^}]*)\}", src):
        bits = [int(x.strip().rstrip("u")) for x in ms.split(",")]
        assert len(set(bits)) == 5 and all(b & (b - 1) == 0 for b in bits)


def test_bench_circuit_compiles(svlib):
    _nvrtc_or_skip()
    n = 30
    g = fused_layered_u3_cz(n, 20, seed=0)
    _, passes, _ = B.sv_plan_info(n, B.SV_C64, g, fuse_max_k=5)
    ns, nc, text = B.sv_jit_check(n, B.SV_C64, g, fuse_max_k=5, compile=True, arch=103)
    assert ns == passes and nc == ns, text[:2000]


@pytest.mark.parametrize("fuse,mode", [(0, 0), (5, 0), (5, 1)])
def test_every_op_kind_compiles(svlib, fuse, mode):
    _nvrtc_or_skip()
    n = 22
    g = random_circuit(n, 160, seed=922, max_controls=3, max_unitary_k=5)
    ns, nc, text = B.sv_jit_check(n, B.SV_C64, g, fuse_max_k=fuse, block_mode=mode, compile=True, arch=103,
                                  tile_qubits=12)
    assert ns > 0 and nc == ns, text[:2000]


def test_mode_validation(svlib):
    with pytest.raises(B.SvError):
        B.sv_jit_set_mode(3)
    B.sv_jit_set_mode(0)
    assert B.sv_jit_info()["mode"] == 0
    B.sv_jit_set_mode(-1)
    assert B.sv_jit_info()["mode"] in (0, 1, 2)


def test_adjoint_template_kernels_compile(svlib):
    """The batched forward and reverse passes of the 20-qubit HEA template
    (checkpoints every two layers) and of a circuit with every generator
    family, controls, bit flips and swaps, and a 3-qubit template (tiles too
    small for register phases: shared-memory phases) all compile."""
    _nvrtc_or_skip()
    from workloads import Gate, hea_ring
    n, layers = 20, 10
    ns, nc, text = B.sv_jit_check_adjoint(n, B.SV_C64, hea_ring(n, layers), 2 * n * layers,
                                          checkpoint_every=6 * n, compile=True)
    assert ns > 0 and nc == ns, text[:2000]
    assert "batch_sweep_body<float, true>" in text and "batch_grad_add<float>" in text
    gates = [Gate("h", [q]) for q in range(6)]
    for i, f in enumerate(["rx", "ry", "rz", "p", "rxx", "ryy", "rzz", "exc1"]):
        k = 2 if f in ("rxx", "ryy", "rzz", "exc1") else 1
        t = [i % 6, (i + 1) % 6][:k]
        c = [(i + 3) % 6] if i % 2 else []
        gates.append(Gate(f, t, c, [i % 2] * len(c), params=[0.0], slots=[i % 3]))
        gates.append(Gate("x", [(i + 2) % 6], [(i + 4) % 6]))
        gates.append(Gate("swap", [i % 6, (i + 5) % 6]))
    gates.append(Gate("exc2", [0, 1, 2, 3], params=[0.0], slots=[1]))
    for dt in (B.SV_C64, B.SV_C128):
        ns, nc, text = B.sv_jit_check_adjoint(6, dt, gates, 3, checkpoint_every=7, compile=True)
        assert ns > 0 and nc == ns, text[:2000]
    ns, nc, text = B.sv_jit_check_adjoint(3, B.SV_C64, hea_ring(3, 2), 12, compile=True)
    assert ns > 0 and nc == ns and "in shared memory" in text, text[:2000]


def test_sources_depend_on_structure_not_angles(svlib):
    """Kernels are kept by program structure: two circuits of the same gates
    at other angles write the same kernel sources (coefficients are read at
    run time), while a circuit of another structure writes others."""
    from workloads import serving_circuit
    n = 24
    a = B.sv_jit_check(n, B.SV_C64, fused_layered_u3_cz(n, 4, seed=11), fuse_max_k=5, compile=False)
    b = B.sv_jit_check(n, B.SV_C64, fused_layered_u3_cz(n, 4, seed=12), fuse_max_k=5, compile=False)
    assert a[0] > 0 and a == b
    c = B.sv_jit_check(n, B.SV_C64, serving_circuit(n, 4, 11), fuse_max_k=5, compile=False)
    assert c[2] != a[2]


# ---- the shared-memory layouts of the compiled passes, executed on the CPU

def _phys(l):
    return l ^ ((l >> 3) & 14)


def _ins0(x, p):
    return ((x >> p) << (p + 1)) | (x & ((1 << p) - 1))


def _xors(block, name, var):
    return [(int(a, 16), int(b, 16)) for a, b in
            re.findall(r"%s \^= \(%s & 0x([0-9a-f]+)u\) \? 0x([0-9a-f]+)u : 0u;" % (name, var), block)]


def _apply(x, start, xs):
    for mask, c in xs:
        if x & mask:
            start ^= c
    return start


def _consts(block, name):
    return [int(v.strip().rstrip('u')) for v in
            re.search(r"const uint32_t %s\[5\] = \{([^}]*)\}" % name, block).group(1).split(',')]


def _phase_maps(block):
    """Local index -> shared-memory slot of a register phase's loads and (if
    it stores to shared memory) stores, from the source's own constants."""
    bits = [int(x) for x in re.search(r"register slots at local bits ([\d ]+)", block).group(1).split()]
    pairs = "true" if bits[0] == 0 else "false"
    assert "reg_load_at<float, 5, %s>" % pairs in block
    stores = "reg_store_at<float, 5, %s>" % pairs in block
    mi, si = _consts(block, "mi"), _xors(block, "si", "tb")
    mo, so = (_consts(block, "mo"), _xors(block, "so", "tb")) if stores else (None, None)
    load, store = {}, ({} if stores else None)
    for tid in range(128):
        tb = tid
        for b in bits:
            tb = _ins0(tb, b)
        for j in range(32):
            l, a = tb, _apply(tb, tb, si)
            c = _apply(tb, tb, so) if stores else None
            for i in range(5):
                if (j >> i) & 1:
                    l |= 1 << bits[i]
                    a ^= mi[i]
                    if stores:
                        c ^= mo[i]
            load[l] = a
            if stores:
                store[l] = c
    return bits[0] == 0, load, store


def _check_pass_layouts(src):
    phys = {l: _phys(l) for l in range(4096)}
    starts = [m.start() for m in re.finditer(r"\{  // phase \d+:", src)] + [len(src)]
    maps = []
    for a, b in zip(starts, starts[1:]):
        block = src[a:b]
        if "register slots" in block:
            maps.append(_phase_maps(block))
        else:  # a shared-memory op phase addresses the tile through phys()
            maps.append((False, phys, phys))
    for pairs, load, store in maps:
        for m in (load, store):
            if m is None:
                continue
            assert sorted(m) == list(range(4096)) and sorted(m.values()) == list(range(4096))
            if pairs:
                assert all(m[l] % 2 == 0 and m[l + 1] == m[l] + 1 for l in range(0, 4096, 2))
    assert maps[0][1] == phys  # the TMA copies leave the stage in the 128-byte swizzle
    for k in range(1, len(maps)):
        assert maps[k - 1][2] == maps[k][1], "phase %d does not load what phase %d stored" % (k, k - 1)
    if "the tile to the state" not in src:
        assert maps[-1][2] is None
        return False
    blk = src[src.index("the tile to the state"):]
    p0 = _xors(blk, "p0", r"gr\.tid")
    pk = [int(x) for x in re.findall(r"s \+ \(p0 \^ (\d+)u\)", blk)]
    assert len(p0) == 7 and len(pk) == 16
    seen = set()
    for tid in range(128):
        base = _apply(tid, 0, p0)
        for k in range(16):
            l = (tid << 1) | (k << 8)
            assert base ^ pk[k] == maps[-1][2][l]
            seen.add(l)
    assert seen == set(range(0, 4096, 2))
    return True


def test_compiled_pass_layouts_are_consistent(svlib):
    """Executes, for every thread and register combination, the shared-memory
    slot arithmetic the generated sources carry: every phase's load and store
    maps are one to one over the tile (16-byte pairs whole and in order), the
    first phase reads the TMA copies' swizzle, each phase reads what the one
    before it stored, and the copy-out reads what the last phase stored
    (every pair once).  Circuits: the 28-qubit layered circuit (heavy passes
    with picked layouts and copy-outs) and a random circuit with wide gates in
    shared-memory phases."""
    cases = [(28, fused_layered_u3_cz(28, 20, seed=0), 5, 0),
             (21, random_circuit(21, 160, seed=921, max_controls=3, max_unitary_k=5), 5, 1)]
    copy_outs = 0
    for n, g, fuse, mode in cases:
        ns, _, src = B.sv_jit_check(n, B.SV_C64, g, fuse_max_k=fuse, block_mode=mode, compile=False,
                                    tile_qubits=12)
        assert ns > 0
        for p in src.split("// ----")[:ns]:
            copy_outs += _check_pass_layouts(p)
    assert copy_outs > 0


def test_generator_store_and_coefficient_choices(svlib):
    """A pass whose last register phase holds local bits 1..4 in registers
    would store each 16-byte pair of a warp to 32 different lines: such passes
    copy the tile out through shared memory instead.  Coefficients at offsets
    known to the generator (rotations, 2x2 blocks, fixed phase tables) come
    from the program in kernel-parameter space (`pc`); only tables whose row
    depends on the thread or the tile read the shared-memory copy (`cf`)."""
    n = 28
    ns, _, src = B.sv_jit_check(n, B.SV_C64, fused_layered_u3_cz(n, 20, seed=0), fuse_max_k=5, compile=False)
    passes = src.split("// ----")[:ns]
    heavy = 0
    for p in passes:
        bits = [[int(x) for x in m.split()] for m in re.findall(r"register slots at local bits ([\d ]+)", p)]
        if {1, 2, 3, 4} <= set(bits[-1]):
            assert "the tile to the state" in p and "reg_store_global" not in p
            heavy += 1
        assert "r_rot<float, 5, " in p and "cf[" not in p  # rotations read pc[...]
        for line in p.splitlines():
            if "r_phase_table<" in line:
                dependent = "tb >>" in line or "base >>" in line
                assert ("(v, cf + " in line) == dependent and ("(v, pc + " in line) != dependent, line
    assert heavy > 0
