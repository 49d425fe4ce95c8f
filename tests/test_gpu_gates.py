"""GPU parity: the CUDA gate kernels (through the C ABI) against the FP64 oracle.

Tolerances (max abs amplitude error vs the oracle): complex128 <= 1e-12 (both
native FP64 and float-float arithmetic), complex64 <= 2e-5.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_00123_gb300 import circuits as C
from paper_2303_00123_gb300.circuits import Gate

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = {"c128": 1e-12, "c128x": 1e-12, "c64": 2e-5}
MODES = ["c128", "c128x", "c64"]


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00123_gb300 import build
    build.build()
    from paper_2303_00123_gb300 import qcgb300
    return qcgb300


def new_state(q, n, mode):
    st = q.State(n, q.C64 if mode == "c64" else q.C128)
    if mode == "c128":
        st.set_arith(q.ARITH_NATIVE)
    elif mode == "c128x":
        st.set_arith(q.ARITH_F32X2)
    return st


def gpu_run(q, n, gates, mode, psi0=None, **kw):
    st = new_state(q, n, mode)
    if psi0 is not None:
        st.from_numpy(psi0)
    st.apply_circuit(gates, **kw)
    out = st.to_numpy().astype(np.complex128)
    st.free()
    return out


def maxerr(a, b):
    return float(np.max(np.abs(a - b)))


def rand_u(rng, d):
    return C.haar_unitary(rng, d)


# ------------------------------------------------------------------ paper examples
@pytest.mark.parametrize("mode", MODES)
def test_worked_index_sets(q, mode):
    """Figs. 2, 3, 6 (n=3): X through qc_apply_c1q swaps exactly the printed pairs."""
    fx = json.load(open(os.path.join(GOLDEN, "index_sets_n3.json")))
    n = fx["n"]
    for case in fx["cases"]:
        st = new_state(q, n, mode)
        st.from_numpy(np.arange(1, (1 << n) + 1).astype(np.complex128))
        st.apply_c1q(np.array([[0, 1], [1, 0]]), case["controls"], case["cstates"], case["target"])
        psi = st.to_numpy().real
        st.free()
        for aj, bj in zip(case["a"], case["b"]):
            assert psi[aj] == bj + 1 and psi[bj] == aj + 1, case["figure"]
        for x in set(range(1 << n)) - set(case["a"]) - set(case["b"]):
            assert psi[x] == x + 1


@pytest.mark.parametrize("mode", MODES)
def test_worked_index_sets_embedded(q, mode):
    """The same index sets with the three qubits of Figs. 2/3/6 embedded in a
    10-qubit register at several positions (exercises the vector kernels)."""
    fx = json.load(open(os.path.join(GOLDEN, "index_sets_n3.json")))
    n = 10
    for place in [(0, 1, 2), (3, 6, 9), (7, 8, 9), (9, 5, 0)]:
        for case in fx["cases"]:
            m = {i: place[i] for i in range(3)}
            st = new_state(q, n, mode)
            st.from_numpy(np.arange(1, (1 << n) + 1).astype(np.complex128))
            st.apply_c1q(np.array([[0, 1], [1, 0]]), [m[c] for c in case["controls"]], case["cstates"],
                         m[case["target"]])
            psi = st.to_numpy().real
            st.free()
            ref = np.arange(1, (1 << n) + 1).astype(np.complex128)
            O.apply_matrix(ref, n, np.array([[0, 1], [1, 0]]), (m[case["target"]],),
                           [m[c] for c in case["controls"]], case["cstates"])
            assert np.array_equal(psi, ref.real), (place, case["figure"])


# ------------------------------------------------------------------ single gates
def one_gate_cases(n, rng):
    """A spread of gates on n qubits: every target, dense / diagonal /
    permutation / exact-phase structures, controls at all positions and
    states, 2-qubit gates on ordered and reversed pairs, k-qubit gates."""
    g = []
    for t in range(n):
        g.append(Gate("U", (t,), matrix=rand_u(rng, 2)))
        g.append(Gate("U", (t,), matrix=rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))))
        for name in ("H", "X", "Y", "Z", "S", "SDG", "T"):
            g.append(Gate(name, (t,)))
        g.append(Gate("P", (t,), theta=float(rng.uniform(-3, 3))))
        g.append(Gate("RZ", (t,), theta=float(rng.uniform(-3, 3))))
        g.append(Gate("RX", (t,), theta=float(rng.uniform(-3, 3))))
        others = [x for x in range(n) if x != t]
        for nc in (1, 2, 3):
            if nc > len(others):
                continue
            cs = [int(v) for v in rng.choice(others, size=nc, replace=False)]
            st = [int(v) for v in rng.integers(0, 2, size=nc)]
            g.append(Gate("U", (t,), controls=cs, cstates=st, matrix=rand_u(rng, 2)))
            g.append(Gate("X", (t,), controls=cs, cstates=st))
            g.append(Gate("P", (t,), controls=cs, cstates=st, theta=float(rng.uniform(-3, 3))))
            g.append(Gate("Z", (t,), controls=cs, cstates=st))
    for a in range(n):
        for b in range(n):
            if a != b and (rng.random() < 0.5 or n <= 6):
                g.append(Gate("U4", (a, b), matrix=rand_u(rng, 4)))
                g.append(Gate("SWAP", (a, b)))
    diag = np.diag(np.exp(1j * rng.uniform(-3, 3, size=4)))
    if n >= 2:
        g.append(Gate("U4", (0, n - 1), matrix=diag))
    if n >= 3:
        g.append(Gate("U4", (n - 1, 1), matrix=np.diag([1, 1, 1, np.exp(0.7j)])))
    for k in (3, 4, 5):
        if k <= n:
            qs = [int(v) for v in rng.choice(n, size=k, replace=False)]
            g.append(Gate("UK", qs, matrix=rand_u(rng, 1 << k)))
    return g


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 9, 12])
def test_single_gates_match_oracle(q, mode, n):
    rng = np.random.default_rng(100 + n)
    phi = C.random_state(n, 200 + n)
    st = new_state(q, n, mode)
    worst = 0.0
    for g in one_gate_cases(n, rng):
        if len(g.qubits) > n:
            continue
        st.from_numpy(phi)
        st.apply_circuit([g])
        got = st.to_numpy().astype(np.complex128)
        ref = phi.copy()
        O.apply_gate(ref, n, g)
        e = maxerr(got, ref)
        worst = max(worst, e)
        assert e <= TOL[mode], (g, e)
    st.free()


@pytest.mark.parametrize("mode", MODES)
def test_direct_entry_points(q, mode):
    """qc_apply_1q / c1q / 2q / kq directly (not through the circuit driver)."""
    n = 8
    rng = np.random.default_rng(5)
    phi = C.random_state(n, 6)
    st = new_state(q, n, mode)
    st.from_numpy(phi)
    ref = phi.copy()
    U = rand_u(rng, 2)
    st.apply_1q(U, 3); O.apply_matrix(ref, n, U, (3,))
    st.apply_c1q(U, [0, 7], [1, 0], 5); O.apply_matrix(ref, n, U, (5,), (0, 7), (1, 0))
    U4 = rand_u(rng, 4)
    st.apply_2q(U4, 6, 1); O.apply_matrix(ref, n, U4, (6, 1))
    U8 = rand_u(rng, 8)
    st.apply_kq(U8, [2, 7, 4], [0], [1]); O.apply_matrix(ref, n, U8, (2, 7, 4), (0,), (1,))
    assert maxerr(st.to_numpy().astype(np.complex128), ref) <= TOL[mode]
    st.free()


# ------------------------------------------------------------------ circuits
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("fuse_k", [0, 2, 3, 4, 5])
def test_random_mix_n12_300_gates(q, mode, fuse_k):
    """n=12, 300 seeded gates (60% Haar U(2), 20% controlled, 20% Haar U(4))
    from |0...0>: final amplitudes against the oracle."""
    n = 12
    gates = C.random_mix(n, 300, seed=0)
    ref = O.run_circuit(n, gates)
    got = gpu_run(q, n, gates, mode, fuse_k=fuse_k)
    assert maxerr(got, ref) <= TOL[mode]


@pytest.mark.parametrize("mode", MODES)
def test_qft_and_brickwork_n14(q, mode):
    n = 14
    x = 5821
    got = gpu_run(q, n, C.qft(n), mode, psi0=O.basis_state(n, x))
    e = np.zeros(1 << n)
    e[x] = 1
    assert maxerr(got, np.fft.fft(e) / math.sqrt(1 << n)) <= TOL[mode]
    gates = C.brickwork(n, 12, seed=3)
    assert maxerr(gpu_run(q, n, gates, mode), O.run_circuit(n, gates)) <= TOL[mode]


@pytest.mark.parametrize("mode", MODES)
def test_graph_capture_and_timing(q, mode):
    import torch
    n = 11
    gates = C.random_mix(n, 80, seed=9)
    ref = O.run_circuit(n, gates)
    st = new_state(q, n, mode)
    s = torch.cuda.Stream()
    st.set_stream(s)
    nl, ms = st.apply_circuit(gates, use_graph=True, time_gates=True)
    assert nl == len(gates) and ms is not None and len(ms) == nl
    assert maxerr(st.to_numpy().astype(np.complex128), ref) <= TOL[mode]
    st.set_basis(0)
    nl, ms = st.apply_circuit(gates, fuse_k=4, time_gates=True)
    assert nl < len(gates) and np.all(ms > 0)
    assert maxerr(st.to_numpy().astype(np.complex128), ref) <= TOL[mode]
    st.free()


def test_wrapped_torch_tensor(q):
    import torch
    n = 10
    t = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    t[0] = 1
    st = q.State.from_tensor(t)
    gates = C.random_mix(n, 50, seed=21)
    st.apply_circuit(gates)
    torch.cuda.synchronize()
    assert maxerr(t.cpu().numpy(), O.run_circuit(n, gates)) <= 1e-12
    st.free()
    assert t.abs().sum().item() > 0   # the borrowed memory is still valid


# ------------------------------------------------------------------ expectation
@pytest.mark.parametrize("mode", MODES)
def test_expectation_values(q, mode):
    n = 10
    psi = C.random_state(n, 31)
    H = C.tfim(n, 0.8) + [(0.3, [("Y", 1), ("X", 3)]), (-0.2, [("Y", 0), ("Z", 2), ("Y", 9)]),
                          (0.5, []), (0.25, [("I", 4)])]
    st = new_state(q, n, mode)
    st.from_numpy(psi)
    ref = O.expect(psi.astype(np.complex64).astype(np.complex128) if mode == "c64" else psi, n, H)
    got = st.expect(H)
    # complex64: exact products of the FP32 amplitudes, float-float sums: 1e-12 * sum |c_t|
    assert abs(got - ref) <= (1e-12 if mode != "c64" else 1e-12 * max(1.0, sum(abs(c) for c, _ in H)))
    st.free()


def test_expectation_closed_forms(q):
    for n in (3, 9):
        st = q.State(n, q.C128)
        H = C.tfim(n, 1.0)
        assert abs(st.expect(H) + (n - 1)) < 1e-13
        st.apply_circuit([Gate("H", (i,)) for i in range(n)])
        assert abs(st.expect(H) + n) < 1e-12
        st.free()


# ------------------------------------------------------------------ errors
def test_invalid_calls_leave_state_unchanged(q):
    n = 6
    phi = C.random_state(n, 1)
    st = q.State(n, q.C128)
    st.from_numpy(phi)
    bad = [
        lambda: st.apply_1q(np.eye(2), 6),
        lambda: st.apply_c1q(np.eye(2), [2], [1], 2),
        lambda: st.apply_c1q(np.eye(2), [1], [2], 0),
        lambda: st.apply_2q(np.eye(4), 3, 3),
        lambda: st.apply_circuit([Gate("H", (0,)), Gate("H", (9,))]),
        lambda: st.apply_circuit([Gate("H", (0,))], fuse_k=9),
        lambda: st.expect([(1.0, [("Q", 0)])]),
        lambda: st.set_basis(1 << n),
    ]
    for f in bad:
        with pytest.raises(q.QCError) as ei:
            f()
        assert ei.value.code == q.QC_ERR_ARG
    assert np.array_equal(st.to_numpy(), phi)
    st.free()


def test_degenerate_cases(q):
    for mode in MODES:
        st = new_state(q, 1, mode)
        st.apply_1q(np.array([[0, 1], [1, 0]]), 0)
        assert np.allclose(st.to_numpy(), [0, 1])
        st.free()
        n = 4
        st = new_state(q, n, mode)
        phi = C.random_state(n, 2)
        st.from_numpy(phi)
        st.apply_1q(np.eye(2), 2)                     # identity: no-op
        st.apply_c1q(np.eye(2), [0, 1, 3], [1, 0, 1], 2)
        assert np.array_equal(st.to_numpy().astype(np.complex128), phi.astype(st.np_dtype).astype(np.complex128))
        st.apply_circuit([])
        U = rand_u(np.random.default_rng(0), 2)
        st.apply_c1q(U, [0, 1, 3], [1, 0, 1], 2)       # all other qubits control
        ref = phi.astype(st.np_dtype).astype(np.complex128)
        O.apply_matrix(ref, n, U, (2,), (0, 1, 3), (1, 0, 1))
        assert maxerr(st.to_numpy().astype(np.complex128), ref) <= TOL[mode]
        st.free()


# ------------------------------------------------------------------ full size
def _sample(t, idx):
    import torch
    return t[torch.as_tensor(idx, device=t.device)].cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("mode", ["c128x", "c128"])
def test_qft_n30_sampled_against_dft(q, mode):
    """n=30 complex128 (17.2 GB), the QFT circuit of Fig. 1 on a seeded basis
    state |x>: 4096 sampled amplitudes against the DFT closed form
    psi_y = exp(-2 pi i x y / 2^n) / 2^(n/2), plus the norm (FP64 reduction)."""
    import torch
    n = 30
    rng = np.random.default_rng(1001)
    x = int(rng.integers(0, 1 << n))
    t = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    st = q.State.from_tensor(t)
    if mode == "c128":
        st.set_arith(q.ARITH_NATIVE)
    st.set_basis(x)
    st.apply_circuit(C.qft(n))
    ys = rng.integers(0, 1 << n, size=4096)
    got = _sample(t, ys)
    ref = np.exp(-2j * np.pi * ((x * ys.astype(object)) % (1 << n)).astype(np.float64) / (1 << n)) / 2 ** (n / 2)
    assert maxerr(got, ref) <= 1e-12
    assert abs(st.expect([(1.0, [])]) - 1.0) <= 1e-12
    st.free()
    del t
    torch.cuda.empty_cache()


def test_brickwork_n30_then_inverse_returns_basis_state(q):
    """n=30 complex128: brickwork (depth 4) followed by its inverse maps |x>
    back to |x> (property valid at any size); sampled amplitudes + norm."""
    import torch
    from tests.test_oracle_pins import _inverse
    n = 30
    rng = np.random.default_rng(1002)
    x = int(rng.integers(0, 1 << n))
    gates = C.brickwork(n, 4, seed=77)
    t = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    st = q.State.from_tensor(t)
    st.set_basis(x)
    st.apply_circuit(gates)
    mid = _sample(t, [x])
    assert abs(mid[0]) < 0.5        # the state really moved away from |x>
    st.apply_circuit(_inverse(gates))
    ys = np.concatenate([[x], rng.integers(0, 1 << n, size=4095)])
    got = _sample(t, ys)
    ref = (ys == x).astype(np.complex128)
    assert maxerr(got, ref) <= 1e-12
    assert abs(st.expect([(1.0, [])]) - 1.0) <= 1e-12
    st.free()
    del t
    torch.cuda.empty_cache()


def test_fused_brickwork_n30_c64_matches_unfused_on_samples(q):
    """n=30 complex64, brickwork depth 6, fused (k=5) vs unfused on the GPU,
    both checked against a product-state closed form at depth 1."""
    import torch
    n = 30
    gates = C.brickwork(n, 6, seed=5)
    outs = []
    rng = np.random.default_rng(3)
    ys = rng.integers(0, 1 << n, size=4096)
    for k in (0, 5):
        t = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
        st = q.State.from_tensor(t)
        st.set_basis(0)
        st.apply_circuit(gates, fuse_k=k)
        outs.append(_sample(t, ys))
        st.free()
        del t
        torch.cuda.empty_cache()
    assert maxerr(outs[0], outs[1]) <= 2e-5
    # depth-1 layer without its CNOTs is a product state: amplitude = prod_q U_q[bit, 0]
    layer = [g for g in C.brickwork(n, 1, seed=5) if not g.controls]
    t = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    st = q.State.from_tensor(t)
    st.set_basis(0)
    st.apply_circuit(layer)
    got = _sample(t, ys)
    ref = np.ones(len(ys), dtype=np.complex128)
    for g in layer:
        bit = (ys >> (n - 1 - g.qubits[0])) & 1
        ref *= g.matrix[bit, 0]
    assert maxerr(got, ref) <= 2e-5
    st.free()


@pytest.mark.parametrize("mode", MODES)
def test_fused_tile_kernel_placements(q, mode):
    """Dense k-qubit blocks (k = 3, 4, 5) through the tile kernel: targets at
    low, high and mixed bit positions, in any order, with and without low and
    high controls, n = 14 and 17 (many tiles; ragged placements)."""
    rng = np.random.default_rng(321)
    for n in (14, 17):
        phi = C.random_state(n, 400 + n)
        st = new_state(q, n, mode)
        cases = [[n - 1, n - 2, n - 3], [0, 1, 2, 3], [n - 1, 0, n // 2, 3, n - 4], [5, 9, 2],
                 [n - 6, n - 5, n - 7, n - 1]]
        for qs in cases:
            for ctl in ([], [n // 3], [n - 1 if n - 1 not in qs else 4], [6, 7]):
                if set(ctl) & set(qs):
                    continue
                cst = [int(v) for v in rng.integers(0, 2, size=len(ctl))]
                U = rand_u(rng, 1 << len(qs))
                st.from_numpy(phi)
                st.apply_kq(U, qs, ctl, cst)
                ref = phi.copy()
                O.apply_matrix(ref, n, U, qs, ctl, cst)
                assert maxerr(st.to_numpy().astype(np.complex128), ref) <= TOL[mode], (n, qs, ctl)
        st.free()


@pytest.mark.parametrize("k", [3, 4, 5])
def test_tensor_core_blocks_match_oracle_and_cuda_cores(q, k):
    """complex64 k-qubit blocks: the tcgen05 path (split TF32) and the FP32
    CUDA-core path both within 2e-5 of the oracle; placements with low and
    high targets, ragged controls; n = 12 (one tile per CTA) and 16."""
    rng = np.random.default_rng(900 + k)
    for n in (12, 16):
        phi = C.random_state(n, 77 + n)
        for trial in range(4):
            qs = [int(v) for v in rng.choice(n, size=k, replace=False)]
            rest = [x for x in range(n) if x not in qs]
            ctl = [int(v) for v in rng.choice(rest, size=trial % 2, replace=False)]
            cst = [1] * len(ctl)
            U = rand_u(rng, 1 << k)
            ref = phi.copy()
            O.apply_matrix(ref, n, U, qs, ctl, cst)
            outs = []
            for tc in (True, False):
                st = q.State(n, q.C64)
                st.set_fused_tc(tc)
                st.from_numpy(phi)
                st.apply_kq(U, qs, ctl, cst)
                outs.append(st.to_numpy().astype(np.complex128))
                st.free()
            for o in outs:
                assert maxerr(o, ref) <= 2e-5, (n, qs, ctl)
            assert maxerr(outs[0], outs[1]) <= 2e-5
    assert q.device_status()["tc_timeouts"] == 0


def test_packed_and_scalar_float_float_are_identical(q):
    """The packed FP32-pair form of the complex128 float-float arithmetic
    performs the same operations in the same order as the scalar form:
    bit-identical states, both within 1e-12 of the oracle."""
    n = 13
    gates = C.random_mix(n, 150, seed=17) + [Gate("RZ", (t,), theta=0.1 * t) for t in range(n)]
    gates += [Gate("P", (3,), controls=(7,), theta=0.77), Gate("U4", (12, 0), matrix=rand_u(np.random.default_rng(1), 4))]
    ref = O.run_circuit(n, gates)
    outs = []
    for packed in (1, 0):
        st = new_state(q, n, "c128x")
        st.set_packed(packed)
        st.apply_circuit(gates)
        outs.append(st.to_numpy())
        st.free()
    assert np.array_equal(outs[0], outs[1])
    assert maxerr(outs[0], ref) <= 1e-12


@pytest.mark.parametrize("n,dtype", [(33, "c128"), (34, "c64")])
def test_maximum_size_states(q, n, dtype):
    """The largest states that fit the GPU's memory (137 GB): a circuit on the
    qubits {0, n/2, n-1} of a seeded basis state |x>.  Amplitudes factorise:
    every other qubit keeps x's bit, and the three active qubits follow the
    oracle's 3-qubit simulation of the same gates (checked on all 8 nonzero
    amplitudes plus sampled zeros), and the norm stays 1."""
    import torch
    a, b, c = 0, n // 2, n - 1
    gates = [Gate("H", (a,)), Gate("X", (c,), controls=(a,)), Gate("U", (b,), matrix=rand_u(np.random.default_rng(3), 2)),
             Gate("P", (b,), controls=(c,), theta=0.61), Gate("U4", (c, a), matrix=rand_u(np.random.default_rng(4), 4)),
             Gate("SWAP", (a, b))]
    remap = {a: 0, b: 1, c: 2}
    small = [Gate(g.name, tuple(remap[t] for t in g.qubits), tuple(remap[t] for t in g.controls), g.cstates,
                  theta=g.theta, matrix=g.matrix) for g in gates]
    rng = np.random.default_rng(33)
    x = int(rng.integers(0, 1 << n))
    bits = lambda v: ((v >> (n - 1 - a)) & 1) * 4 + ((v >> (n - 1 - b)) & 1) * 2 + ((v >> (n - 1 - c)) & 1)
    ref3 = O.run_circuit(3, small, O.basis_state(3, bits(x)))
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    t = torch.zeros(1 << n, dtype=tdt, device="cuda")
    st = q.State.from_tensor(t)
    st.set_basis(x)
    st.apply_circuit(gates)
    mask = (1 << (n - 1 - a)) | (1 << (n - 1 - b)) | (1 << (n - 1 - c))
    ys, ref = [], []
    for r in range(8):
        y = (x & ~mask) | (((r >> 2) & 1) << (n - 1 - a)) | (((r >> 1) & 1) << (n - 1 - b)) | ((r & 1) << (n - 1 - c))
        ys.append(y)
        ref.append(ref3[r])
    for _ in range(64):                           # amplitudes that must stay zero
        y = int(rng.integers(0, 1 << n))
        if (y & ~mask) != (x & ~mask):
            ys.append(y)
            ref.append(0.0)
    got = t[torch.as_tensor(ys, device="cuda")].cpu().numpy().astype(np.complex128)
    assert maxerr(got, np.array(ref)) <= (1e-12 if dtype == "c128" else 2e-5)
    assert abs(st.expect([(1.0, [])]) - 1.0) <= (1e-12 if dtype == "c128" else 1e-5)
    st.free()
    del t
    torch.cuda.empty_cache()


@pytest.mark.parametrize("mode", MODES)
def test_fused_qft_with_linear_phase_runs(q, mode):
    """QFT with fusion: each stage's controlled phases run as one linear-phase
    sweep; against the DFT and the oracle, n = 6, 13, 17 (phase bits in and
    above a vector, anchors at every position)."""
    for n in (6, 13, 17):
        x = (0x5A5A5 * 7 + n) % (1 << n)
        got = gpu_run(q, n, C.qft(n), mode, psi0=O.basis_state(n, x), fuse_k=4)
        e = np.zeros(1 << n)
        e[x] = 1
        assert maxerr(got, np.fft.fft(e) / math.sqrt(1 << n)) <= TOL[mode], n
    # runs with scattered linear qubits, a theta0 term and a Z, on a random state
    n = 11
    rng = np.random.default_rng(8)
    gates = [Gate("H", (q_,)) for q_ in range(n)]
    gates += [Gate("P", (4,), controls=(int(c),), theta=float(rng.uniform(-3, 3))) for c in (0, 9, 2, 10, 7, 5, 1)]
    gates += [Gate("P", (4,), theta=0.37), Gate("Z", (6,), controls=(4,)), Gate("U", (3,), matrix=rand_u(rng, 2))]
    gates += [Gate("P", (int(t),), controls=(8,), theta=float(rng.uniform(-3, 3))) for t in (0, 10, 3, 2)]
    phi = C.random_state(n, 5)
    assert maxerr(gpu_run(q, n, gates, mode, psi0=phi, fuse_k=3), O.run_circuit(n, gates, phi)) <= TOL[mode]


# ------------------------------------------------------------------ TFXY Trotter circuit
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("fuse_k", [0, 2, 3, 5])
def test_tfxy_trotter_n13(q, mode, fuse_k):
    """The Hamiltonian-simulation circuit of Sec. 4 (3 Trotter steps, seeded
    angles) on a random 13-qubit state, gate by gate and fused (complex64
    blocks of k >= 3 on the tensor cores), against the oracle."""
    n = 13
    gates = C.tfxy_trotter(n, 3, seed=5)
    phi = C.random_state(n, 6)
    assert maxerr(gpu_run(q, n, gates, mode, psi0=phi, fuse_k=fuse_k), O.run_circuit(n, gates, phi)) <= TOL[mode]


@pytest.mark.parametrize("dtype,fuse_k", [("c128", 2), ("c64", 5)])
def test_tfxy_n28_then_inverse_returns_basis_state(q, dtype, fuse_k):
    """n=28: two fused Trotter steps then their inverse map |x> back to |x>
    (a property valid at any size); sampled amplitudes."""
    import torch
    from tests.test_oracle_pins import _inverse
    n = 28
    rng = np.random.default_rng(2801)
    x = int(rng.integers(0, 1 << n))
    gates = C.tfxy_trotter(n, 2, seed=9)
    t = torch.zeros(1 << n, dtype=torch.complex128 if dtype == "c128" else torch.complex64, device="cuda")
    st = q.State.from_tensor(t)
    st.set_basis(x)
    st.apply_circuit(gates, fuse_k=fuse_k)
    assert abs(_sample(t, [x])[0]) < 0.9          # the state moved
    st.apply_circuit(_inverse(gates), fuse_k=fuse_k)
    ys = np.concatenate([[x], rng.integers(0, 1 << n, size=4095)])
    got = _sample(t, ys)
    ref = (ys == x).astype(np.complex128)
    assert maxerr(got, ref) <= (1e-12 if dtype == "c128" else 2e-5)
    st.free()
    del t
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ OpenQASM programs
@pytest.mark.parametrize("mode", MODES)
def test_qasm_program_through_the_library(q, mode):
    """A program written as OpenQASM 2.0 (QFT + two TFXY Trotter steps, n=12),
    read back and applied gate by gate and fused, against the oracle on the
    original gate list."""
    n = 12
    gates = C.qft(n) + C.tfxy_trotter(n, 2, seed=3)
    m, back, _ = q.qasm_parse(q.qasm_write(n, gates))
    assert m == n and len(back) == len(gates)
    phi = C.random_state(n, 12)
    ref = O.run_circuit(n, gates, phi)
    for k in (0, 4):
        assert maxerr(gpu_run(q, n, back, mode, psi0=phi, fuse_k=k), ref) <= TOL[mode]


@pytest.mark.parametrize("n", [2, 3, 5, 8, 13])
def test_two_qubit_chain_sums_match_oracle(q, n):
    """complex128 dense 2-qubit gates in the default arithmetic (fixed-binade
    product chains): every ordered pair of qubits at n <= 5 (sampled pairs
    above), Haar matrices and general (non-unitary) matrices scaled to norm 1,
    on a random state; 1e-12 against the oracle, and within 1e-12 of the
    TwoSum form (packed mode 1)."""
    rng = np.random.default_rng(600 + n)
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b]
    if len(pairs) > 24:
        pairs = [pairs[i] for i in rng.choice(len(pairs), size=24, replace=False)]
    gates = []
    for a, b in pairs:
        gates.append(Gate("U4", (a, b), matrix=rand_u(rng, 4)))
        m = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
        gates.append(Gate("U4", (b, a), matrix=m / np.linalg.norm(m, 2)))
    phi = C.random_state(n, 601)
    ref = O.run_circuit(n, gates, phi)
    outs = []
    for mode in (2, 1):
        st = new_state(q, n, "c128x")
        st.set_packed(mode)
        st.from_numpy(phi)
        st.apply_circuit(gates)
        outs.append(st.to_numpy())
        st.free()
    assert maxerr(outs[0], ref) <= 1e-12
    assert maxerr(outs[0], outs[1]) <= 1e-12
