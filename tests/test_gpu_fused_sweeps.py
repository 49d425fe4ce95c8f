"""GPU parity for the merged sweeps of fused circuits, against the FP64 oracle.

* A 1-qubit gate on qubit a followed by a run of phase gates that all involve
  a (a QFT stage, Fig. 1) runs as one sweep (k_dense_linphase): U on the
  anchor pair, then exp(i phi) on its anchor-1 member.  Cases put the anchor
  at several bit positions (4 and up) and the linear qubits inside the
  thread's window (in-vector and run bits) and above it, with and without a
  phase on the anchor itself.
* A run of SWAPs on disjoint pairs runs as one bit permutation (k_permute):
  tiles of 2^t contiguous amplitudes plus the bits the permutation brings into
  them, paired tiles exchanged in place.  Cases cover pairs among the low
  bits, pairs linking low and high bits, pairs among high bits only, and the
  full bit reversal of the QFT.

Tolerances as in the other gate tests: complex128 1e-12, complex64 2e-5
(max abs amplitude error).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_00123_gb300 import circuits as C
from paper_2303_00123_gb300.circuits import Gate

pytestmark = pytest.mark.gpu

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


def run(q, n, gates, mode, psi0, fuse_k=2):
    st = q.State(n, q.C64 if mode == "c64" else q.C128)
    if mode == "c128":
        st.set_arith(q.ARITH_NATIVE)
    elif mode == "c128x":
        st.set_arith(q.ARITH_F32X2)
    st.from_numpy(psi0)
    st.apply_circuit(gates, fuse_k=fuse_k)
    out = st.to_numpy().astype(np.complex128)
    st.free()
    return out


def stage(rng, n, a, controls, theta0=None):
    """Haar U(2) on qubit a, then controlled phases on a from `controls`."""
    g = [Gate("U", (a,), matrix=C.haar_unitary(rng, 2))]
    for c in controls:
        g.append(Gate("P", (a,), controls=(int(c),), theta=float(rng.uniform(-math.pi, math.pi))))
    if theta0 is not None:
        g.append(Gate("P", (a,), theta=theta0))
    return g


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [6, 9, 13, 16])
def test_hadamard_and_phase_run_in_one_sweep(q, mode, n):
    rng = np.random.default_rng(300 + n)
    gates = []
    # anchors from qubit 0 (highest bit) to qubit n-5 (bit 4, the lowest merged)
    for a in sorted({0, 1, n // 2 - 1, n - 5}):
        others = [c for c in range(n) if c != a]
        lows = [c for c in others if c >= n - 4]                 # bits 0..3: inside the window
        highs = [c for c in others if c < n - 4]
        ctl = list(rng.choice(lows, size=min(2, len(lows)), replace=False)) + \
            list(rng.choice(highs, size=min(5, len(highs)), replace=False))
        gates += stage(rng, n, a, ctl, theta0=0.4 if a % 2 else None)
    plan = q.fuse_plan(n, gates, 2)
    merged = [e for e in plan if e[0] == "phase" and e[4] is not None]
    assert len(merged) >= 2
    phi = C.random_state(n, n)
    assert np.max(np.abs(run(q, n, gates, mode, phi) - O.run_circuit(n, gates, phi))) <= TOL[mode]


def disjoint_pairs(rng, qubits, k):
    qs = list(rng.permutation(qubits))[: 2 * k]
    return [(int(qs[2 * i]), int(qs[2 * i + 1])) for i in range(k)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [4, 5, 8, 12, 15])
def test_disjoint_swap_runs_as_one_permutation(q, mode, n):
    rng = np.random.default_rng(400 + n)
    phi = C.random_state(n, 40 + n)
    cases = [
        [(i, n - 1 - i) for i in range(n // 2)],                        # bit reversal
        disjoint_pairs(rng, range(n), n // 2),                          # random
        disjoint_pairs(rng, range(max(0, n - 6), n), min(3, n // 2)),   # low bits only
        disjoint_pairs(rng, range(0, n - 6), 2) if n >= 10 else [(0, 1), (n - 1, n - 2)],  # high / mixed
    ]
    for pairs in cases:
        if len(pairs) < 2:
            continue
        gates = [Gate("SWAP", p) for p in pairs] + [Gate("H", (0,))]
        plan = q.fuse_plan(n, gates, 2)
        assert plan[0][0] == "swap", pairs
        got = run(q, n, gates, mode, phi)
        assert np.max(np.abs(got - O.run_circuit(n, gates, phi))) <= TOL[mode], pairs


@pytest.mark.parametrize("mode", ["c128x", "c64"])
def test_fused_qft_n30_sampled_against_dft(q, mode):
    """n=30, the QFT of Fig. 1 with fusion (26 merged H + phase sweeps, 2
    phase runs, one 2-qubit block, one bit-reversal permutation) on a seeded
    basis state |x>: 4096 sampled amplitudes against
    psi_y = exp(-2 pi i x y / 2^n) / 2^(n/2), plus the norm."""
    import torch
    n = 30
    rng = np.random.default_rng(3001)
    x = int(rng.integers(0, 1 << n))
    t = torch.zeros(1 << n, dtype=torch.complex64 if mode == "c64" else torch.complex128, device="cuda")
    st = q.State.from_tensor(t)
    st.set_basis(x)
    nl = st.apply_circuit(C.qft(n), fuse_k=2)
    ys = rng.integers(0, 1 << n, size=4096)
    got = t[torch.as_tensor(ys, device=t.device)].cpu().numpy().astype(np.complex128)
    ref = np.exp(-2j * np.pi * ((x * ys.astype(object)) % (1 << n)).astype(np.float64) / (1 << n)) / 2 ** (n / 2)
    assert np.max(np.abs(got - ref)) <= TOL[mode]
    assert abs(st.expect([(1.0, [])]) - 1.0) <= (1e-12 if mode != "c64" else 1e-5)
    st.free()
    del t
    torch.cuda.empty_cache()
