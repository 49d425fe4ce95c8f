"""GPU parity of the adjoint-gradient path against the FP64 oracle's
parameter-shift gradients and energies.

Tolerances: complex128 sweeps: energies and gradients <= 1e-10 absolute;
complex64 sweeps with FP64 reductions: <= 2e-4 absolute.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_00123_gb300 import circuits as C
from paper_2303_00123_gb300.circuits import Gate

pytestmark = pytest.mark.gpu
TOL = {"c128": 1e-10, "c128x": 1e-10, "c64": 2e-4}


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00123_gb300 import build
    build.build()
    from paper_2303_00123_gb300 import qcgb300
    return qcgb300


def dt(q, mode):
    return {"c128": (q.C128, q.ARITH_NATIVE), "c128x": (q.C128, q.ARITH_F32X2), "c64": (q.C64, q.ARITH_AUTO)}[mode]


def with_thetas(gates, th):
    out, k = [], 0
    for g in gates:
        if g.name in ("RX", "RY", "RZ") and not g.controls:
            g = Gate(g.name, g.qubits, theta=float(th[k]))
            k += 1
        out.append(g)
    return out


@pytest.mark.parametrize("mode", ["c128", "c128x", "c64"])
def test_single_rotation_closed_form(q, mode):
    d, a = dt(q, mode)
    ths = np.linspace(-3.0, 3.0, 9)[:, None]
    for name, H in (("RY", [(1.0, [("Z", 0)])]), ("RX", [(1.0, [("Z", 0)])])):
        e, g = q.adjoint_grad(1, [Gate(name, (0,), theta=0.0)], H, ths, dtype=d, arith=a)
        assert np.max(np.abs(e - np.cos(ths[:, 0]))) <= TOL[mode]          # <Z> = cos(theta)
        assert np.max(np.abs(g[:, 0] + np.sin(ths[:, 0]))) <= TOL[mode]    # d/dtheta = -sin(theta)
    e, g = q.adjoint_grad(1, [Gate("H", (0,)), Gate("RZ", (0,), theta=0.0)], [(1.0, [("X", 0)])], ths,
                          dtype=d, arith=a)
    assert np.max(np.abs(e - np.cos(ths[:, 0]))) <= TOL[mode]
    assert np.max(np.abs(g[:, 0] + np.sin(ths[:, 0]))) <= TOL[mode]


@pytest.mark.parametrize("mode", ["c128", "c128x", "c64"])
def test_hea_against_parameter_shift(q, mode):
    d, a = dt(q, mode)
    n, layers, B = 6, 3, 4
    th = C.hea_thetas(n, layers, seed=3, batch=B)
    template = C.hea(n, layers, th[0])
    H = C.tfim(n, 1.0)
    e, g = q.adjoint_grad(n, template, H, th, dtype=d, arith=a)
    assert g.shape == (B, 2 * n * layers)
    for b in range(B):
        gates = C.hea(n, layers, th[b])
        assert abs(e[b] - O.energy(n, gates, H)) <= TOL[mode]
        assert np.max(np.abs(g[b] - O.param_shift_grad(n, gates, H))) <= TOL[mode]


@pytest.mark.parametrize("mode", ["c128x", "c64"])
def test_general_circuit_against_parameter_shift(q, mode):
    """Rotations about all axes mixed with controlled and 2-qubit gates, a
    Hamiltonian with Y terms, and controls at every position."""
    d, a = dt(q, mode)
    n = 7
    rng = np.random.default_rng(8)
    gates = []
    for layer in range(3):
        for t in range(n):
            gates.append(Gate(["RX", "RY", "RZ"][(t + layer) % 3], (t,), theta=float(rng.uniform(-3, 3))))
        gates.append(Gate("U4", (layer, n - 1 - layer), matrix=C.haar_unitary(rng, 4)))
        gates.append(Gate("X", (2,), controls=(5, 0), cstates=(1, 0)))
        gates.append(Gate("P", (3,), controls=(6,), theta=0.4))
        gates.append(Gate("RZ", (1,), controls=(4,), theta=0.9))      # controlled rotation: not a parameter
    H = C.tfim(n, 0.6) + [(0.3, [("Y", 1), ("Y", 2)]), (-0.7, [("X", 0), ("Y", 4), ("Z", 6)]), (0.2, [])]
    P = q.count_params(gates)
    assert P == 3 * n
    th = np.array([[g.theta for g in gates if g.name in ("RX", "RY", "RZ") and not g.controls]])
    e, g = q.adjoint_grad(n, gates, H, th, dtype=d, arith=a)
    assert abs(e[0] - O.energy(n, gates, H)) <= TOL[mode]
    ps = O.param_shift_grad(n, gates, H)
    assert np.max(np.abs(g[0] - ps)) <= TOL[mode]


@pytest.mark.parametrize("mode", ["c64", "c128x"])
def test_full_size_hea_sampled(q, mode):
    """n=20, 10 layers (400 parameters), TFIM h=1.0: batch of 64 (complex64)
    or 4 (complex128); energies of two sets and three sampled gradient
    entries against the oracle (energy and parameter shift)."""
    d, a = dt(q, mode)
    n, layers = 20, 10
    B = 64 if mode == "c64" else 4
    th = C.hea_thetas(n, layers, seed=2025, batch=B)
    H = C.tfim(n, 1.0)
    e, g = q.adjoint_grad(n, C.hea(n, layers, th[0]), H, th, dtype=d, arith=a)
    assert e.shape == (B,) and g.shape == (B, 400)
    for b in (0, B - 1):
        assert abs(e[b] - O.energy(n, C.hea(n, layers, th[b]), H)) <= TOL[mode]
    gates = C.hea(n, layers, th[B - 1])
    pidx = O.parametric_indices(gates)
    for k in (0, 217, 399):
        i = pidx[k]
        t = gates[i].theta
        gp = [Gate(x.name, x.qubits, x.controls, x.cstates, theta=(t + math.pi / 2 if j == i else x.theta))
              for j, x in enumerate(gates)]
        gm = [Gate(x.name, x.qubits, x.controls, x.cstates, theta=(t - math.pi / 2 if j == i else x.theta))
              for j, x in enumerate(gates)]
        ps = 0.5 * (O.energy(n, gp, H) - O.energy(n, gm, H))
        assert abs(g[B - 1, k] - ps) <= TOL[mode], (k, g[B - 1, k], ps)


def test_autograd_function(q):
    import torch
    from paper_2303_00123_gb300.autograd import energy
    n, layers = 5, 2
    th0 = C.hea_thetas(n, layers, seed=9, batch=3)
    gates = C.hea(n, layers, th0[0])
    H = C.tfim(n, 1.0)
    th = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    E = energy(th, gates, H, n, dtype=q.C128)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    (E * w).sum().backward()
    for b in range(3):
        gb = C.hea(n, layers, th0[b])
        assert abs(E[b].item() - O.energy(n, gb, H)) <= 1e-10
        assert np.max(np.abs(th.grad[b].numpy() - w[b].item() * O.param_shift_grad(n, gb, H))) <= 1e-10


def test_adjoint_argument_errors(q):
    H = C.tfim(3, 1.0)
    with pytest.raises(q.QCError):
        q.adjoint_grad(3, [Gate("UK", (0, 1, 2), matrix=np.eye(8))], H, None)
    with pytest.raises(q.QCError):
        q.adjoint_grad(3, [Gate("RX", (5,), theta=0.1)], H, None)
    with pytest.raises(q.QCError):
        q.adjoint_grad(3, [Gate("RX", (0,), theta=0.1)], [(1.0, [("Z", 7)])], None)
