"""Excitation gates (Sec. 4.2 gate table: single excitation / Givens and
double excitation) on the GPU against the oracle: forward application
(fused and unfused, with controls) and adjoint gradients of both, the double
excitation's also against the four-term shift rule."""
import numpy as np
import pytest

import oracle
import paper_2608_09733_gb300 as sv
from paper_2608_09733_gb300.binding import SvError
from workloads import Gate, Term, random_circuit

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _circuit(n, seed, count=80):
    rng = np.random.default_rng(seed)
    g = random_circuit(n, 50, seed=seed)
    for _ in range(count):
        q = [int(x) for x in rng.permutation(n)[:5]]
        if rng.random() < 0.5:
            g.append(Gate("exc1", q[:2], params=[rng.uniform(0, 6.3)],
                          controls=[q[2]] if rng.random() < 0.2 else []))
        else:
            g.append(Gate("exc2", q[:4], params=[rng.uniform(0, 6.3)]))
    return g


@pytest.mark.parametrize("dtype,tol", [(sv.SV_C64, 2e-6), (sv.SV_C128, 1e-12)])
@pytest.mark.parametrize("n", [6, 16, 21])
@pytest.mark.parametrize("fuse", [0, 5])
def test_excitation_circuits_match_oracle(svlib, cuda_dev, dtype, tol, n, fuse):
    g = _circuit(n, n)
    st = torch.empty(2 ** n, dtype=torch.complex64 if dtype == sv.SV_C64 else torch.complex128, device="cuda")
    sv.sv_init_basis(st, 0)
    sv.sv_apply_circuit(st, g, fuse_max_k=fuse)
    assert np.abs(st.cpu().numpy() - oracle.run(n, g)).max() < tol


@pytest.mark.parametrize("dtype,tol", [(sv.SV_C64, 1e-4), (sv.SV_C128, 1e-10)])
def test_exc1_adjoint_gradients_match_oracle(svlib, cuda_dev, dtype, tol):
    n, batch = 8, 3
    gates, slot = [Gate("x", [q]) for q in (0, 2, 5)], 0
    for layer in range(3):
        for a in range(n - 1):
            gates.append(Gate("exc1", [a, a + 1], slots=[slot]))
            slot += 1
        gates.append(Gate("rz", [layer], slots=[slot]))
        slot += 1
    H = [Term("ZZ", [0, 1], 0.5), Term("XX", [2, 3], -0.3), Term("YY", [2, 3], -0.3), Term("Z", [7], 0.9)]
    params = np.random.default_rng(1).uniform(0, 2 * np.pi, size=(batch, slot))
    val, grad = sv.sv_adjoint_grad(n, dtype, gates, params, H)
    for b in range(batch):
        rv, rg = oracle.adjoint_grad(n, gates, params[b], H, slot)
        assert abs(val[b] - rv) < tol and np.abs(grad[b] - rg).max() < tol


def _exc2_template(n, rng):
    """EXC2 rotations (some controlled, one with a control on |0>) among
    EXC1 and RZ, a literal-angle EXC2 and a shared slot."""
    gates, slot = [Gate("x", [q]) for q in (0, 1, 4)], 0
    for layer in range(2):
        for a in range(0, n - 3, 2):
            q = [a, a + 1, a + 2, a + 3]
            ctrl = [(a + 5) % n] if (a + layer) % 3 == 0 and (a + 5) % n not in q else []
            gates.append(Gate("exc2", q, ctrl, [layer % 2] * len(ctrl), slots=[slot]))
            slot += 1
        gates.append(Gate("exc1", [layer, layer + 2], slots=[slot]))
        slot += 1
        gates.append(Gate("rz", [n - 1 - layer], slots=[slot]))
        slot += 1
    gates.append(Gate("exc2", [n - 1, 0, 2, 5], params=[0.7]))  # literal angle: a fixed gate
    gates.append(Gate("exc2", [1, 3, 5, 6], slots=[0]))          # slot 0 shared
    return gates, slot


@pytest.mark.parametrize("dtype,tol", [(sv.SV_C64, 1e-4), (sv.SV_C128, 1e-10)])
def test_exc2_adjoint_gradients_match_oracle(svlib, cuda_dev, dtype, tol):
    """The double excitation's gradient on the GPU (Sec. 4.2: generator Y on
    the exchanged pair) against the oracle's adjoint, with checkpoints."""
    n, batch = 8, 3
    rng = np.random.default_rng(11)
    gates, slot = _exc2_template(n, rng)
    H = [Term("ZZ", [0, 1], 0.5), Term("XX", [2, 3], -0.3), Term("YY", [4, 5], 0.4), Term("Z", [7], 0.9),
         Term("X", [6], 0.2)]
    params = rng.uniform(0, 2 * np.pi, size=(batch, slot))
    for ck in (0, 5):
        val, grad = sv.sv_adjoint_grad(n, dtype, gates, params, H, checkpoint_every=ck)
        for b in range(batch):
            rv, rg = oracle.adjoint_grad(n, gates, params[b], H, slot)
            assert abs(val[b] - rv) < tol and np.abs(grad[b] - rg).max() < tol, (ck, b)


def test_exc2_gradient_matches_four_term_shift_rule(svlib, cuda_dev):
    """Uncontrolled EXC2 gradients against the paper's four-term shift rule
    (shifts +-pi/2, +-3pi/2; the generator spectrum is {-1, 0, 1})."""
    n = 7
    rng = np.random.default_rng(12)
    gates = [Gate("h", [q]) for q in range(n)]
    slot = 0
    for a in range(3):
        gates.append(Gate("exc2", [a, a + 2, a + 1, a + 4], slots=[slot]))
        gates.append(Gate("ry", [a + 3], slots=[slot + 1]))
        slot += 2
    H = [Term("ZZ", [q, q + 1], 1.0) for q in range(n - 1)] + [Term("X", [q], 0.7) for q in range(n)]
    th = rng.uniform(0, 2 * np.pi, size=(1, slot))
    ps = oracle.param_shift_grad(n, gates, th[0], H, slot)
    _, g128 = sv.sv_adjoint_grad(n, sv.SV_C128, gates, th, H)
    _, g64 = sv.sv_adjoint_grad(n, sv.SV_C64, gates, th, H)
    assert np.abs(g128[0] - ps).max() < 1e-10
    assert np.abs(g64[0] - ps).max() < 1e-4


def test_exc2_with_too_many_controls_is_rejected_by_the_adjoint(svlib, cuda_dev):
    g = [Gate("exc2", [0, 1, 2, 3], [4, 5, 6], slots=[0])]
    with pytest.raises(SvError):
        sv.sv_adjoint_grad(7, sv.SV_C64, g, np.zeros((1, 1)), [Term("Z", [0], 1.0)])
