"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics (no GPU).  Each test names the passage or the closed form it uses.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_00123_gb300 import circuits as C
from paper_2303_00123_gb300.circuits import Gate

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PAULI = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


def kron_all(factors):
    out = np.array([[1.0 + 0j]])
    for f in factors:
        out = np.kron(out, f)
    return out


def rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def dense_gate(n, U, qubits, controls=(), cstates=()):
    """Dense 2^n x 2^n matrix of a (controlled) gate built only from Kronecker
    products (Eq. (1)): sum over matrix entries U[r,c] of the outer products
    |r_i><c_i| on each target qubit, identity elsewhere; the control
    condition enters as the projector |s><s| on each control qubit."""
    k = len(qubits)
    dim = 1 << k
    N = 1 << n
    act = np.zeros((N, N), dtype=complex)
    for r in range(dim):
        for c in range(dim):
            if U[r, c] == 0:
                continue
            fac = [PAULI["I"]] * n
            for i, q in enumerate(qubits):
                ri, ci = (r >> (k - 1 - i)) & 1, (c >> (k - 1 - i)) & 1
                e = np.zeros((2, 2), dtype=complex)
                e[ri, ci] = 1
                fac[q] = e
            for q, s in zip(controls, cstates):
                p = np.zeros((2, 2), dtype=complex)
                p[s, s] = 1
                fac[q] = p
            act += U[r, c] * kron_all(fac)
    if controls:
        fac = [PAULI["I"]] * n
        for q, s in zip(controls, cstates):
            p = np.zeros((2, 2), dtype=complex)
            p[s, s] = 1
            fac[q] = p
        act += np.eye(N) - kron_all(fac)   # identity where the controls do not match
    return act


# ----------------------------------------------------------- Figs. 2, 3, 6
def test_index_sets_of_the_worked_examples():
    """The pairs (a_j, b_j) that a (controlled) 1-qubit gate mixes, n=3,
    against the index sets printed in Figs. 2, 3 and 6."""
    fx = json.load(open(os.path.join(GOLDEN, "index_sets_n3.json")))
    n = fx["n"]
    for case in fx["cases"]:
        psi = np.arange(1, (1 << n) + 1).astype(complex)
        O.apply_matrix(psi, n, PAULI["X"], (case["target"],), case["controls"], case["cstates"])
        a, b = case["a"], case["b"]
        for aj, bj in zip(a, b):
            assert psi[aj] == bj + 1 and psi[bj] == aj + 1, case["figure"]
        untouched = sorted(set(range(1 << n)) - set(a) - set(b))
        for x in untouched:
            assert psi[x] == x + 1, case["figure"]
        if "mR" in case:   # Fig. 2 masks: m_R = 2^(n-q-1) - 1, m_L = 2^(n-1) - 1 - m_R
            q = case["target"]
            assert case["mR"] == (1 << (n - q - 1)) - 1
            assert case["mL"] == (1 << (n - 1)) - 1 - case["mR"]
            # a_j = (j & m_R) + ((j & m_L) << 1) reproduces the printed sets
            assert [(j & case["mR"]) + ((j & case["mL"]) << 1) for j in range(4)] == a


def test_paper_specialisations_of_pauli_gates():
    """Sec. 2.1: X swaps the pair, Y gives (-i phi_b, i phi_a), Z negates b."""
    rng = np.random.default_rng(1)
    n = 4
    for q in range(n):
        phi = rand_c(rng, 1 << n)
        s = 1 << (n - q - 1)
        a = [x for x in range(1 << n) if not x & s]
        b = [x + s for x in a]
        for name, fa, fb in (("X", lambda pa, pb: pb, lambda pa, pb: pa),
                             ("Y", lambda pa, pb: -1j * pb, lambda pa, pb: 1j * pa),
                             ("Z", lambda pa, pb: pa, lambda pa, pb: -pb)):
            psi = phi.copy()
            O.apply_gate(psi, n, Gate(name, (q,)))
            np.testing.assert_array_equal(psi[a], fa(phi[a], phi[b]))
            np.testing.assert_array_equal(psi[b], fb(phi[a], phi[b]))


# ----------------------------------------------------------- Eq. (1)
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_one_qubit_gate_equals_kronecker_product(n):
    """psi = (I_l (x) U (x) I_r) phi with I_l of size 2^q (Eq. (1), Def. 1)."""
    rng = np.random.default_rng(10 + n)
    for q in range(n):
        U = rand_c(rng, 2, 2)                 # general, non-symmetric
        phi = rand_c(rng, 1 << n)
        ref = np.kron(np.kron(np.eye(1 << q), U), np.eye(1 << (n - q - 1))) @ phi
        psi = phi.copy()
        O.apply_matrix(psi, n, U, (q,))
        np.testing.assert_allclose(psi, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_controlled_gates_equal_kronecker_construction(n):
    rng = np.random.default_rng(20 + n)
    for _ in range(12):
        nc = int(rng.integers(1, min(3, n - 1) + 1))
        qs = rng.choice(n, size=nc + 1, replace=False)
        t, ctrl = int(qs[0]), [int(v) for v in qs[1:]]
        st = [int(v) for v in rng.integers(0, 2, size=nc)]
        U = rand_c(rng, 2, 2)
        phi = rand_c(rng, 1 << n)
        ref = dense_gate(n, U, (t,), ctrl, st) @ phi
        psi = phi.copy()
        O.apply_matrix(psi, n, U, (t,), ctrl, st)
        np.testing.assert_allclose(psi, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_two_qubit_gates_equal_kronecker_construction(n):
    """Sec. 2.3 on any (also non-adjacent, also reversed) pair; U4's index is
    2*bit(q0) + bit(q1) (the order Eq. (1) fixes)."""
    rng = np.random.default_rng(30 + n)
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b]
    for q0, q1 in pairs:
        U = rand_c(rng, 4, 4)
        phi = rand_c(rng, 1 << n)
        ref = dense_gate(n, U, (q0, q1)) @ phi
        psi = phi.copy()
        O.apply_matrix(psi, n, U, (q0, q1))
        np.testing.assert_allclose(psi, ref, rtol=0, atol=1e-12)
    # adjacent pair in increasing order is exactly I_l (x) U4 (x) I_r
    for q in range(n - 1):
        U = rand_c(rng, 4, 4)
        phi = rand_c(rng, 1 << n)
        ref = np.kron(np.kron(np.eye(1 << q), U), np.eye(1 << (n - q - 2))) @ phi
        psi = phi.copy()
        O.apply_matrix(psi, n, U, (q, q + 1))
        np.testing.assert_allclose(psi, ref, rtol=0, atol=1e-12)


def test_k_qubit_and_controlled_two_qubit_gates():
    rng = np.random.default_rng(40)
    n = 6
    for k in (3, 4):
        for _ in range(4):
            qs = [int(v) for v in rng.choice(n, size=k, replace=False)]
            U = rand_c(rng, 1 << k, 1 << k)
            phi = rand_c(rng, 1 << n)
            psi = phi.copy()
            O.apply_matrix(psi, n, U, qs)
            np.testing.assert_allclose(psi, dense_gate(n, U, qs) @ phi, rtol=0, atol=1e-11)
    qs = [int(v) for v in rng.choice(n, size=4, replace=False)]
    U = rand_c(rng, 4, 4)
    phi = rand_c(rng, 1 << n)
    psi = phi.copy()
    O.apply_matrix(psi, n, U, qs[:2], qs[2:], (0, 1))
    np.testing.assert_allclose(psi, dense_gate(n, U, qs[:2], qs[2:], (0, 1)) @ phi, rtol=0, atol=1e-12)


def test_invalid_gates_are_rejected():
    psi = O.basis_state(3)
    with pytest.raises(ValueError):
        O.apply_matrix(psi, 3, np.eye(2), (3,))
    with pytest.raises(ValueError):
        O.apply_matrix(psi, 3, np.eye(2), (1,), (1,), (1,))
    with pytest.raises(ValueError):
        O.apply_matrix(psi, 3, np.eye(4), (0, 0))


# ----------------------------------------------------------- closed forms
def test_bell_and_ghz_states():
    psi = O.run_circuit(2, [Gate("H", (0,)), Gate("X", (1,), controls=(0,))])
    np.testing.assert_allclose(psi, np.array([1, 0, 0, 1]) / math.sqrt(2), atol=1e-15)
    for n in (3, 5, 8):
        gates = [Gate("H", (0,))] + [Gate("X", (q,), controls=(q - 1,)) for q in range(1, n)]
        psi = O.run_circuit(n, gates)
        ref = np.zeros(1 << n, dtype=complex)
        ref[0] = ref[-1] = 1 / math.sqrt(2)
        np.testing.assert_allclose(psi, ref, atol=1e-15)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 8, 10])
def test_qft_of_basis_state_is_the_dft(n):
    """Fig. 1's QFT circuit maps |x> to the unitary DFT of e_x (library FFT)."""
    rng = np.random.default_rng(50 + n)
    for x in set([0, (1 << n) - 1] + [int(v) for v in rng.integers(0, 1 << n, size=4)]):
        psi = O.run_circuit(n, C.qft(n), O.basis_state(n, x))
        e = np.zeros(1 << n)
        e[x] = 1
        np.testing.assert_allclose(psi, np.fft.fft(e) / math.sqrt(1 << n), atol=1e-13)


def _inverse(gates):
    inv = []
    for g in reversed(gates):
        name = g.name.upper()
        if name in ("U", "U4", "UK"):
            inv.append(Gate(name, g.qubits, g.controls, g.cstates, matrix=np.conj(np.asarray(g.matrix)).T))
        elif name in ("P", "RX", "RY", "RZ"):
            inv.append(Gate(name, g.qubits, g.controls, g.cstates, theta=-g.theta))
        elif name in ("S", "T"):
            inv.append(Gate(name + "DG", g.qubits, g.controls, g.cstates))
        elif name in ("SDG", "TDG"):
            inv.append(Gate(name[:-2], g.qubits, g.controls, g.cstates))
        else:
            inv.append(g)   # H, X, Y, Z, SWAP are self-inverse
    return inv


def test_norm_preservation_and_inverse_circuit():
    n = 8
    phi = C.random_state(n, 7)
    gates = C.random_mix(n, 200, seed=3) + C.qft(n) + C.brickwork(n, 3, seed=4)
    psi = O.run_circuit(n, gates, phi)
    assert abs(np.linalg.norm(psi) - 1) < 1e-13
    back = O.run_circuit(n, _inverse(gates), psi)
    np.testing.assert_allclose(back, phi, atol=1e-13)


def test_haar_inputs_are_unitary():
    rng = np.random.default_rng(0)
    for d in (2, 4, 8):
        U = C.haar_unitary(rng, d)
        np.testing.assert_allclose(U.conj().T @ U, np.eye(d), atol=1e-14)


# ----------------------------------------------------------- expectation values
def test_tfim_expectation_closed_forms():
    for n in (2, 4, 7):
        H = C.tfim(n, 1.0)
        assert abs(O.expect(O.basis_state(n), n, H) + (n - 1)) < 1e-13       # <0|H|0> = -(n-1)
        plus = O.run_circuit(n, [Gate("H", (q,)) for q in range(n)])
        assert abs(O.expect(plus, n, H) + n) < 1e-12                          # <+|H|+> = -n


def test_expectation_equals_dense_matrix_form():
    n = 5
    rng = np.random.default_rng(60)
    psi = C.random_state(n, 61)
    H = C.tfim(n, 0.7) + [(0.3, [("Y", 1), ("X", 3)]), (-0.2, [("Y", 0), ("Z", 2), ("Y", 4)])]
    dense = np.zeros((1 << n, 1 << n), dtype=complex)
    for c, ops in H:
        fac = [PAULI["I"]] * n
        for letter, q in ops:
            fac[q] = PAULI[letter]
        dense += c * kron_all(fac)
    assert abs(O.expect(psi, n, H) - np.vdot(psi, dense @ psi).real) < 1e-13


def test_rotation_gate_closed_forms():
    for t in np.linspace(-3, 3, 7):
        g = [Gate("RY", (0,), theta=float(t))]
        H = [(1.0, [("Z", 0)])]
        assert abs(O.energy(1, g, H) - math.cos(t)) < 1e-14                  # <Z> = cos(theta)
        assert abs(O.param_shift_grad(1, g, H)[0] + math.sin(t)) < 1e-14     # d/dtheta = -sin(theta)
        gx = [Gate("RX", (0,), theta=float(t))]
        assert abs(O.energy(1, gx, H) - math.cos(t)) < 1e-14
        gz = [Gate("H", (0,)), Gate("RZ", (0,), theta=float(t))]
        assert abs(O.energy(1, gz, [(1.0, [("X", 0)])]) - math.cos(t)) < 1e-14


def test_parameter_shift_matches_analytic_derivative_and_finite_differences():
    """Parameter shift against (a) the analytic derivative of exp(-i theta P/2),
    dU/dtheta = -(i/2) P U, evaluated with dense matrices, and (b) central
    finite differences with h = 1e-4 (O(h^2) ~ 1e-8 truncation)."""
    n, layers = 3, 2
    th = C.hea_thetas(n, layers, seed=70)
    gates = C.hea(n, layers, th)
    H = C.tfim(n, 1.0)
    ps = O.param_shift_grad(n, gates, H)
    fd = O.finite_diff_grad(n, gates, H, h=1e-4)
    np.testing.assert_allclose(ps, fd, atol=1e-7)
    dense_H = np.zeros((1 << n, 1 << n), dtype=complex)
    for c, ops in H:
        fac = [PAULI["I"]] * n
        for letter, q in ops:
            fac[q] = PAULI[letter]
        dense_H += c * kron_all(fac)
    mats = [dense_gate(n, O.gate_matrix(g), g.qubits, g.controls, g.cstates) for g in gates]
    psi0 = O.basis_state(n)
    idx = O.parametric_indices(gates)
    for k, i in enumerate(idx):
        g = gates[i]
        P = kron_all([PAULI[g.name[1]] if q == g.qubits[0] else PAULI["I"] for q in range(n)])
        left = psi0.copy()
        for m in mats[:i + 1]:
            left = m @ left
        dpsi = -0.5j * P @ left
        for m in mats[i + 1:]:
            dpsi = m @ dpsi
        psi = O.run_circuit(n, gates)
        analytic = 2 * np.vdot(psi, dense_H @ dpsi).real
        assert abs(ps[k] - analytic) < 1e-12


def test_generators_follow_their_recipes():
    n = 6
    q = C.qft(n)
    assert len(q) == n + n * (n - 1) // 2 + n // 2
    b = C.brickwork(n, 4, seed=1)
    assert len(b) == 4 * n + 2 * 3 + 2 * 2          # even layers: 3 CNOTs, odd: 2
    assert len(C.brickwork(30, 40, seed=0)) == 1780   # 1200 U(2) + 580 CNOT
    m = C.random_mix(12, 300, seed=0)
    kinds = [("U4" if g.name == "U4" else "C" if g.controls else "U") for g in m]
    assert 0.5 < kinds.count("U") / 300 < 0.7 and 0.1 < kinds.count("C") / 300 < 0.3
    h = C.hea(4, 3, C.hea_thetas(4, 3, seed=2))
    assert len(O.parametric_indices(h)) == 2 * 4 * 3


def test_tfxy_block_is_a_product_of_two_qubit_exponentials():
    """Each block of the TFXY Trotter circuit (Sec. 4 figure): CNOT(i -> j),
    RX(a) on i, RZ(b) on j, CNOT(i -> j) equals exp(-i a/2 X_i X_j)
    exp(-i b/2 Z_i Z_j) -- conjugation by the CNOT maps X_i to X_i X_j and Z_j
    to Z_i Z_j.  Checked against matrix exponentials (scipy) on a 4-qubit
    state for an adjacent and a distant pair."""
    from scipy.linalg import expm
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)
    n = 4
    rng = np.random.default_rng(31)
    for i, j in ((1, 2), (3, 0)):
        a, b = rng.uniform(-math.pi, math.pi, size=2)
        block = [Gate("X", (j,), controls=(i,), cstates=(1,)), Gate("RX", (i,), theta=a),
                 Gate("RZ", (j,), theta=b), Gate("X", (j,), controls=(i,), cstates=(1,))]

        def two(A, B):          # A on qubit i, B on qubit j, identity elsewhere (qubit 0 = MSB)
            ops = [np.eye(2, dtype=complex)] * n
            ops[i], ops[j] = A, B
            m = ops[0]
            for o in ops[1:]:
                m = np.kron(m, o)
            return m
        U = expm(-0.5j * a * two(X, X)) @ expm(-0.5j * b * two(Z, Z))
        phi = C.random_state(n, 40 + i)
        np.testing.assert_allclose(O.run_circuit(n, block, phi), U @ phi, atol=1e-13)


def test_tfxy_layout_follows_the_figure():
    """Two Trotter steps on four qubits: RZ layer, blocks on pairs (0,1) and
    (2,3), RZ layer, block on (1,2) -- twice; 40 gates."""
    g = C.tfxy_trotter(4, 2, seed=0)
    assert len(g) == 40
    sig = [(x.name, x.qubits, tuple(x.controls)) for x in g[:20]]
    rz = lambda qs: [("RZ", (q,), ()) for q in qs]
    blk = lambda i, j: [("X", (j,), (i,)), ("RX", (i,), ()), ("RZ", (j,), ()), ("X", (j,), (i,))]
    assert sig == rz(range(4)) + blk(0, 1) + blk(2, 3) + rz(range(4)) + blk(1, 2)
    assert [(x.name, x.qubits, tuple(x.controls)) for x in g[20:]] == sig


# ----------------------------------------------------------- named gate matrices
# The entries below are written out here, independently of oracle.gate_matrix:
# Sec. 2.1's Clifford+T gates (S = diag(1, i), T = diag(1, e^{i pi/4})), the
# Hadamard, and the readings P(theta) = diag(1, e^{i theta}),
# R_P(theta) = exp(-i theta P / 2) of the gates the paper's circuits use.
_R2 = 1.0 / math.sqrt(2.0)
WRITTEN = {
    "H": [[_R2, _R2], [_R2, -_R2]],
    "X": [[0, 1], [1, 0]],
    "Y": [[0, -1j], [1j, 0]],
    "Z": [[1, 0], [0, -1]],
    "S": [[1, 0], [0, 1j]],
    "SDG": [[1, 0], [0, -1j]],
    "T": [[1, 0], [0, _R2 + 1j * _R2]],
    "TDG": [[1, 0], [0, _R2 - 1j * _R2]],
}


@pytest.mark.parametrize("name", sorted(WRITTEN))
def test_fixed_gates_act_as_their_written_matrices(name):
    """Every placement on a random 4-qubit state against I (x) M (x) I with
    M's entries typed in above: a transposed, conjugated or mis-angled entry
    (T = diag(1, e^{i pi/8}), S = diag(1, -i), ...) fails."""
    M = np.array(WRITTEN[name], dtype=complex)
    n = 4
    rng = np.random.default_rng(80)
    for q in range(n):
        phi = rand_c(rng, 1 << n)
        psi = phi.copy()
        O.apply_gate(psi, n, Gate(name, (q,)))
        ref = np.kron(np.kron(np.eye(1 << q), M), np.eye(1 << (n - q - 1))) @ phi
        np.testing.assert_allclose(psi, ref, rtol=0, atol=1e-14)


def test_clifford_t_relations():
    """T^2 = S, S^2 = Z, S^dag S = T^dag T = I, H Z H = X, applied with the
    oracle to a random state (each side a gate sequence)."""
    n = 3
    phi = C.random_state(n, 81)
    rel = [(["T", "T"], ["S"]), (["S", "S"], ["Z"]), (["S", "SDG"], []), (["SDG", "S"], []),
           (["T", "TDG"], []), (["TDG", "T"], []), (["H", "Z", "H"], ["X"]), (["T"] * 4, ["Z"])]
    for lhs, rhs in rel:
        for q in range(n):
            a = O.run_circuit(n, [Gate(g, (q,)) for g in lhs], phi)
            b = O.run_circuit(n, [Gate(g, (q,)) for g in rhs], phi)
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-15, err_msg="%s = %s" % (lhs, rhs))


@pytest.mark.parametrize("name", ["RX", "RY", "RZ"])
def test_rotations_are_exponentials_of_paulis(name):
    """R_P(theta) = exp(-i theta P / 2) (reading C5) against a library matrix
    exponential of the Pauli matrix typed in this file, for angles of both
    signs -- a transposed rotation is R_P(-theta) and fails."""
    from scipy.linalg import expm
    P = PAULI[name[1]]
    n = 3
    rng = np.random.default_rng(82)
    for t in (-2.5, -0.7, 0.3, 1.9, math.pi):
        for q in range(n):
            phi = rand_c(rng, 1 << n)
            psi = phi.copy()
            O.apply_gate(psi, n, Gate(name, (q,), theta=t))
            M = expm(-0.5j * t * P)
            ref = np.kron(np.kron(np.eye(1 << q), M), np.eye(1 << (n - q - 1))) @ phi
            np.testing.assert_allclose(psi, ref, rtol=0, atol=1e-14)


def test_rotation_amplitudes_on_basis_states():
    """Amplitude by amplitude: RY(t)|0> = cos(t/2)|0> + sin(t/2)|1>,
    RX(t)|0> = cos(t/2)|0> - i sin(t/2)|1>, RZ(t)|1> = e^{i t/2}|1>,
    P(t)|1> = e^{i t}|1>."""
    for t in (-2.0, -0.4, 0.9, 2.7):
        c, s = math.cos(t / 2), math.sin(t / 2)
        np.testing.assert_allclose(O.run_circuit(1, [Gate("RY", (0,), theta=t)]), [c, s], atol=1e-15)
        np.testing.assert_allclose(O.run_circuit(1, [Gate("RX", (0,), theta=t)]), [c, -1j * s], atol=1e-15)
        np.testing.assert_allclose(O.run_circuit(1, [Gate("RZ", (0,), theta=t)], O.basis_state(1, 1)),
                                   [0, complex(c, s)], atol=1e-15)
        np.testing.assert_allclose(O.run_circuit(1, [Gate("RZ", (0,), theta=t)]), [complex(c, -s), 0], atol=1e-15)
        np.testing.assert_allclose(O.run_circuit(1, [Gate("P", (0,), theta=t)], O.basis_state(1, 1)),
                                   [0, complex(math.cos(t), math.sin(t))], atol=1e-15)
