"""GPU parity for complex128 fused blocks on the tensor cores (k_fused_tc128).

A dense k-qubit block (k = 3..5) on a complex128 state with float-float
arithmetic runs as one GEMM per 128-group tile on fp16 tensor cores: each
state entry is rounded to 48 bits against its group's largest exponent and cut
into six base-2^8 digits, each matrix entry into seven, and the digit products
are accumulated by level in exact FP32 integer sums.  These
cases compare it with the FP64 oracle at the complex128 tolerance (1e-12 max
abs) and with the CUDA-core float-float path, on states whose groups mix
large, tiny and zero amplitudes, on an unnormalised vector (amplitudes up to
~50, as in an adjoint co-state), and for block placements with targets and
controls below, inside and above the tile's low bits.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_00123_gb300 import circuits as C
from paper_2303_00123_gb300.circuits import Gate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00123_gb300 import build
    build.build()
    from paper_2303_00123_gb300 import qcgb300
    return qcgb300


def run(q, n, gates, psi0, fuse_k, tc=True):
    st = q.State(n, q.C128)
    st.set_arith(q.ARITH_F32X2)
    st.set_fused_tc(tc)
    st.from_numpy(psi0)
    st.apply_circuit(gates, fuse_k=fuse_k)
    out = st.to_numpy()
    st.free()
    return out


def block(rng, qubits, controls=(), cstates=None):
    k = len(qubits)
    return Gate("UK" if k > 2 else ("U4" if k == 2 else "U"), tuple(qubits), controls=tuple(controls),
                cstates=tuple(cstates) if cstates is not None else tuple(1 for _ in controls),
                matrix=C.haar_unitary(rng, 1 << k))


@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("n", [12, 14])
def test_dense_blocks_against_oracle(q, k, n):
    rng = np.random.default_rng(700 + 10 * n + k)
    placements = [list(range(k)), list(range(n - k, n)), sorted(rng.choice(n, size=k, replace=False).tolist())]
    gates = [block(rng, p) for p in placements]
    gates.append(block(rng, placements[2], controls=[c for c in range(n) if c not in placements[2]][:1]))
    phi = C.random_state(n, 3)
    got = run(q, n, gates, phi, fuse_k=k)
    ref = O.run_circuit(n, gates, phi)
    assert np.max(np.abs(got - ref)) <= 1e-12
    assert np.max(np.abs(got - run(q, n, gates, phi, fuse_k=k, tc=False))) <= 1e-12


@pytest.mark.parametrize("k", [3, 5])
def test_groups_with_large_tiny_and_zero_amplitudes(q, k):
    """Per-group scaling: amplitudes spanning 1e-30 .. 50, exact zeros, and a
    group that is all zero; the result is compared in absolute terms."""
    n = 13
    rng = np.random.default_rng(90 + k)
    phi = C.random_state(n, 9)
    phi[::7] *= 1e-30
    phi[::11] = 0.0
    phi[:64] = 0.0
    phi[100:140] *= 50.0
    gates = [block(rng, sorted(rng.choice(n, size=k, replace=False).tolist())) for _ in range(3)]
    got = run(q, n, gates, phi, fuse_k=k)
    ref = O.run_circuit(n, gates, phi)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(phi)))


def test_fused_brickwork_and_tfxy_n16(q):
    n = 16
    phi = C.random_state(n, 4)
    for gates in (C.brickwork(n, 8, seed=5), C.tfxy_trotter(n, 2, seed=6)):
        ref = O.run_circuit(n, gates, phi)
        for k in (3, 4, 5):
            assert np.max(np.abs(run(q, n, gates, phi, fuse_k=k) - ref)) <= 1e-12


def test_non_unitary_block_through_the_kq_entry_point(q):
    """qc_apply_kq takes any matrix: entries up to ~40 (the digit scale of the
    matrix follows its largest entry) and a tiny-norm matrix."""
    n = 12
    rng = np.random.default_rng(55)
    phi = C.random_state(n, 5)
    for scale in (37.0, 3e-9):
        M = scale * (rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32)))
        g = [Gate("UK", (1, 4, 6, 9, 11), matrix=M)]
        st = q.State(n, q.C128)
        st.set_arith(q.ARITH_F32X2)
        st.from_numpy(phi)
        st.apply_kq(M, [1, 4, 6, 9, 11])
        got = st.to_numpy()
        st.free()
        ref = O.run_circuit(n, g, phi)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_brickwork_n30_tensor_cores_match_gate_by_gate(q):
    """Full size (n=30, 17.2 GB): brickwork depth 40 fused into 5-qubit blocks on
    the tensor cores against the same circuit applied gate by gate (float-float
    CUDA-core sweeps), compared over the whole state on the device; the norm
    stays 1."""
    import torch
    n = 30
    gates = C.brickwork(n, 40, seed=2001)
    x = 987654321 % (1 << n)
    out = []
    for fuse_k in (0, 5):
        t = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
        st = q.State.from_tensor(t)
        st.set_arith(q.ARITH_F32X2)
        st.set_fused_tc(True)
        st.set_basis(x)
        st.apply_circuit(gates, fuse_k=fuse_k)
        st.free()
        out.append(t)
    diff = 0.0
    for a, b in zip(out[0].split(1 << 26), out[1].split(1 << 26)):
        diff = max(diff, float(torch.max(torch.abs(a - b))))
    norm = float(torch.linalg.vector_norm(out[1]))
    del out
    torch.cuda.empty_cache()
    assert diff <= 1e-12, diff
    assert abs(norm - 1.0) <= 1e-12, norm
