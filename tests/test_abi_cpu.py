"""C-ABI checks that need no GPU: the library builds, loads and exports every
function declared in include/qcgb300.h; argument validation; and the host-side
fusion planner, pinned through the FP64 oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def q():
    from paper_2303_00123_gb300 import build
    build.build()
    from paper_2303_00123_gb300 import qcgb300
    return qcgb300


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "qcgb300.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qc_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(q):
    names = declared_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(q.lib, name), name
    assert q.version().startswith("qcgb300")


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_argument_validation_without_gpu(q):
    h = ctypes.c_void_p()
    assert q.lib.qc_state_alloc(0, q.C128, ctypes.byref(h)) == q.QC_ERR_ARG
    assert q.lib.qc_state_alloc(5, 7, ctypes.byref(h)) == q.QC_ERR_ARG
    assert q.lib.qc_state_alloc(5, q.C128, None) == q.QC_ERR_ARG
    assert q.lib.qc_state_free(None) == q.QC_OK
    assert q.lib.qc_apply_1q(None, None, 0) == q.QC_ERR_ARG
    assert b"NULL" in q.lib.qc_last_error()
    if not _has_gpu():
        # no device: a valid request fails cleanly with QC_ERR_CUDA, no fallback
        assert q.lib.qc_state_alloc(5, q.C128, ctypes.byref(h)) == q.QC_ERR_CUDA


def test_fuse_plan_rejects_bad_gates(q):
    from paper_2303_00123_gb300.circuits import Gate
    with pytest.raises(q.QCError):
        q.fuse_plan(3, [Gate("H", (3,))], 0)
    with pytest.raises(q.QCError):
        q.fuse_plan(3, [Gate("X", (1,), controls=(1,))], 0)
    with pytest.raises(q.QCError):
        q.fuse_plan(3, [Gate("H", (0,))], 6)


@pytest.mark.parametrize("fuse_k", [0, 2, 3, 4, 5])
def test_fusion_plan_reproduces_the_circuit(q, fuse_k):
    """Applying the planned blocks with the oracle equals applying the original
    gates with the oracle (fusion may only change rounding)."""
    from oracle import oracle as O
    from paper_2303_00123_gb300 import circuits as C
    n = 7
    gates = C.random_mix(n, 120, seed=11) + C.qft(n) + C.brickwork(n, 4, seed=12)
    gates += [C.Gate("X", (2,), controls=(0, 5), cstates=(1, 0)), C.Gate("RZ", (3,), theta=0.3)]
    plan = q.fuse_plan(n, gates, fuse_k)
    if fuse_k >= 2:
        assert len(plan) < (0.6 if fuse_k == 2 else 0.35) * len(gates)
        assert max(len(b[0]) + len(b[1]) for b in plan if b[0] not in ("phase", "swap")) <= max(fuse_k, 3)
    else:
        assert len(plan) == len(gates)
    phi = C.random_state(n, 13)
    ref = O.run_circuit(n, gates, phi)
    psi = phi.copy()
    apply_plan(O, psi, n, plan)
    np.testing.assert_allclose(psi, ref, atol=1e-12)


def apply_plan(O, psi, n, plan):
    """Apply a fusion plan with the oracle; a linear phase run is applied as
    the gates it stands for: its 2x2 matrix on the anchor, if any, then P(theta)
    on the anchor, controlled."""
    swap = np.eye(4)[[0, 2, 1, 3]]
    for entry in plan:
        if entry[0] == "swap":
            for a, b in entry[1]:
                O.apply_matrix(psi, n, swap, (a, b))
            continue
        if entry[0] == "phase":
            _, anchor, lin, theta0, pre = entry
            if pre is not None:
                O.apply_matrix(psi, n, pre, (anchor,))
            P = lambda t: np.diag([1, np.exp(1j * t)])
            if theta0 != 0:
                O.apply_matrix(psi, n, P(theta0), (anchor,))
            for qb, t in lin:
                O.apply_matrix(psi, n, P(t), (anchor,), (qb,), (1,))
        else:
            qubits, controls, cstates, U = entry
            O.apply_matrix(psi, n, U, qubits, controls, cstates)


def test_qft_phase_runs_are_fused():
    """Each QFT stage's controlled phases (Fig. 1) share the stage's target and
    become one linear-phase launch; the plan reproduces the circuit."""
    from oracle import oracle as O
    from paper_2303_00123_gb300 import build, circuits as C
    build.build()
    from paper_2303_00123_gb300 import qcgb300 as q
    for n in (5, 9):
        gates = C.qft(n) + [C.Gate("Z", (1,)), C.Gate("S", (1,), controls=(3,)), C.Gate("T", (1,))]
        plan = q.fuse_plan(n, gates, 3)
        runs = [e for e in plan if e[0] == "phase"]
        assert len(runs) >= n - 2
        phi = C.random_state(n, 21)
        psi = phi.copy()
        apply_plan(O, psi, n, plan)
        np.testing.assert_allclose(psi, O.run_circuit(n, gates, phi), atol=1e-12)


def test_fusion_of_brickwork_reduces_sweeps(q):
    from paper_2303_00123_gb300 import circuits as C
    g = C.brickwork(30, 40, seed=0)
    counts = {k: len(q.fuse_plan(30, g, k)) for k in (0, 2, 3, 4, 5)}
    assert counts[0] == 1780
    assert counts[5] < counts[4] < counts[3] < counts[2] < counts[0]


@pytest.mark.parametrize("fuse_k", [3, 4, 5])
def test_partial_block_emission_reproduces_the_circuit(q, fuse_k):
    """When a gate would widen a block past k qubits the planner emits only the
    fullest touched blocks and keeps growing the rest: deep brickwork, Trotter
    and random circuits exercise that path; the oracle applies plan and gates."""
    from oracle import oracle as O
    from paper_2303_00123_gb300 import circuits as C
    n = 10
    for gates in (C.brickwork(n, 12, seed=31), C.tfxy_trotter(n, 3, seed=32), C.random_mix(n, 200, seed=33)):
        plan = q.fuse_plan(n, gates, fuse_k)
        phi = C.random_state(n, 34)
        psi = phi.copy()
        apply_plan(O, psi, n, plan)
        np.testing.assert_allclose(psi, O.run_circuit(n, gates, phi), atol=1e-12)


def _mixed_circuit(n, ngates, seed):
    """Random gates of every kind the planner treats differently: dense 1q and
    2q, (doubly) controlled gates with control states 0/1, runs of disjoint SWAPs,
    runs of controlled phases sharing a qubit, named gates."""
    from paper_2303_00123_gb300 import circuits as C
    from paper_2303_00123_gb300.circuits import Gate
    rng = np.random.default_rng(seed)
    g = []
    while len(g) < ngates:
        r = rng.random()
        qs = [int(v) for v in rng.choice(n, size=min(n, 4), replace=False)]
        if r < 0.3:
            g.append(Gate("U", (qs[0],), matrix=C.haar_unitary(rng, 2)))
        elif r < 0.45:
            g.append(Gate("U4", (qs[0], qs[1]), matrix=C.haar_unitary(rng, 4)))
        elif r < 0.6:
            g.append(Gate("X", (qs[0],), controls=(qs[1],), cstates=(int(rng.integers(2)),)))
        elif r < 0.7 and n >= 3:
            g.append(Gate("U", (qs[0],), controls=(qs[1], qs[2]), cstates=(int(rng.integers(2)), 1),
                          matrix=C.haar_unitary(rng, 2)))
        elif r < 0.8 and n >= 4:
            g.append(Gate("SWAP", (qs[0], qs[1])))
            g.append(Gate("SWAP", (qs[2], qs[3])))
        elif r < 0.9:
            for other in qs[1:]:
                g.append(Gate("P", (qs[0],), controls=(other,), theta=float(rng.uniform(-3, 3))))
        else:
            g.append(Gate(["H", "S", "T", "RX", "RY", "RZ"][int(rng.integers(6))], (qs[0],),
                          theta=float(rng.uniform(-3, 3))))
    return g


@pytest.mark.parametrize("seed", range(12))
def test_fusion_plans_of_random_mixed_circuits(q, seed):
    """Property: for random mixed circuits (n = 4..7) and every fusion width,
    the planned entries applied with the oracle equal the circuit applied gate
    by gate, and no dense block exceeds the width."""
    from oracle import oracle as O
    from paper_2303_00123_gb300 import circuits as C
    n = 4 + seed % 4
    gates = _mixed_circuit(n, 60, 500 + seed)
    phi = C.random_state(n, 600 + seed)
    ref = O.run_circuit(n, gates, phi)
    for k in (2, 3, 4, 5):
        plan = q.fuse_plan(n, gates, k)
        for b in plan:
            if b[0] not in ("phase", "swap") and len(b[0]) + len(b[1]) > max(k, 3):
                raise AssertionError("block wider than k=%d: %r" % (k, (b[0], b[1])))
        psi = phi.copy()
        apply_plan(O, psi, n, plan)
        np.testing.assert_allclose(psi, ref, atol=1e-12, err_msg="k=%d" % k)


def test_fusion_block_counts_at_n30(q):
    """Sweeps the planner makes for the n=30 workloads (each block is one pass over
    the state): brickwork depth 40 and TFXY 10 steps at k=5."""
    from paper_2303_00123_gb300 import circuits as C
    assert len(q.fuse_plan(30, C.brickwork(30, 40, seed=2001), 5)) <= 150
    assert len(q.fuse_plan(30, C.tfxy_trotter(30, 10, seed=1003), 5)) <= 80


def test_count_params(q):
    from paper_2303_00123_gb300 import circuits as C
    n, layers = 5, 3
    gates = C.hea(n, layers, C.hea_thetas(n, layers, seed=1))
    assert q.count_params(gates) == 2 * n * layers
    gates.append(C.Gate("RZ", (1,), controls=(2,), theta=0.3))   # controlled: not a parameter
    assert q.count_params(gates) == 2 * n * layers


def test_expect_pass_counts(q):
    """qc_expect's pass planning (host only): the TFIM chain's X terms on the
    qubits above a tile's low bits need ceil((n - m) / h) passes with m = 3
    low bits and h = 9 generators (tiles of 2^12 amplitudes, both dtypes);
    states that fit one tile need one pass; one long string needs one pass;
    an empty sum none."""
    from paper_2303_00123_gb300 import circuits as C
    for n in (1, 5, 12, 13, 19, 20, 26, 30, 34):
        for dt, m, L in ((q.C128, 3, 12), (q.C64, 3, 12)):
            want = 1 if n <= L else -(-(n - m) // (L - m))
            assert q.expect_passes(n, dt, C.tfim(n, 1.0)) == want, (n, dt)
    assert q.expect_passes(30, q.C128, [(1.0, [("X", i) for i in range(30)])]) == 1
    assert q.expect_passes(30, q.C128, [(1.0, [("Z", i) for i in range(30)])]) == 1
    assert q.expect_passes(30, q.C128, []) == 0
    with pytest.raises(q.QCError):
        q.expect_passes(30, q.C128, [(1.0, [("X", 30)])])


def test_qft_plan_merges_hadamards_and_swaps(q):
    """QFT (Fig. 1) at n=30 with fusion: each stage's H joins its phase run
    (anchors up to qubit n-5), the last stages fuse into a 2-qubit block, and
    the 15 final SWAPs become one bit permutation."""
    from paper_2303_00123_gb300 import circuits as C
    n = 30
    plan = q.fuse_plan(n, C.qft(n), 2)
    runs = [e for e in plan if e[0] == "phase"]
    swaps = [e for e in plan if e[0] == "swap"]
    assert len(swaps) == 1 and sorted(swaps[0][1]) == [(i, n - 1 - i) for i in range(n // 2)]
    assert sum(e[4] is not None for e in runs) == n - 4
    assert all(e[4] is None for e in runs if e[1] > n - 5)
    assert len(plan) == 1 + len(runs) + 2 + 1      # runs, H(26), H(27), block(28, 29), permutation


def test_swap_runs_need_disjoint_pairs(q):
    """Only SWAPs on disjoint pairs merge; a qubit seen twice starts a new run,
    and a single SWAP stays a matrix block."""
    from oracle import oracle as O
    from paper_2303_00123_gb300 import circuits as C
    n = 8
    gates = [C.Gate("SWAP", (0, 5)), C.Gate("SWAP", (1, 7)), C.Gate("SWAP", (5, 2)), C.Gate("SWAP", (3, 4)),
             C.Gate("H", (0,)), C.Gate("SWAP", (6, 1))]
    plan = q.fuse_plan(n, gates, 2)
    kinds = [e[0] if isinstance(e[0], str) else "matrix" for e in plan]
    assert kinds == ["swap", "swap", "matrix", "matrix"]
    assert plan[0][1] == [(0, 5), (1, 7)] and plan[1][1] == [(5, 2), (3, 4)]
    phi = C.random_state(n, 5)
    psi = phi.copy()
    apply_plan(O, psi, n, plan)
    np.testing.assert_allclose(psi, O.run_circuit(n, gates, phi), atol=1e-12)
