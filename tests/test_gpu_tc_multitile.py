"""GPU parity of the tensor-core block kernels where every CTA runs several tiles.

A fused dense block on k = 3..5 qubits runs on the tensor cores one 128-group
tile at a time (complex64: split-TF32 products; complex128: exact fp16 digit
slices); a CTA loads its next tile while the MMAs of the current one run,
flips its mbarrier phase per tile and reuses its tensor memory.  At n = 22..24
a block has 2^(n-k-7) tiles (up to 2^14) for a grid of one or two CTAs per SM,
so these cases exercise the second and later tiles of every CTA.  Each is
compared element by element with the FP64 oracle (Eq. (1), Sec. 2.4) at the
amplitude tolerances: 1e-12 (complex128), 2e-5 (complex64).

The wait-limit test runs the time-out path of both kernels (the one-role
kernel and the warp-specialised pipeline): with a limit of zero polls the
first wait gives up, the kernel waits for the MMAs it committed before
freeing its tensor memory, and the next synchronising call reports
QC_ERR_TIMEOUT; the context stays usable.
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


def block(rng, qubits, controls=(), cstates=None):
    k = len(qubits)
    return Gate("UK", tuple(qubits), controls=tuple(controls),
                cstates=tuple(cstates) if cstates is not None else tuple(1 for _ in controls),
                matrix=C.haar_unitary(rng, 1 << k))


def placements(rng, n, k):
    """Targets at the lowest bit positions, at the highest, spread at random,
    and a random set with one control (state 0) -- each one block."""
    mixed = sorted(rng.choice(n, size=k, replace=False).tolist())
    rest = [c for c in range(n) if c not in mixed]
    ctl = int(rng.choice(rest))
    return [block(rng, list(range(n - k, n))), block(rng, list(range(k))), block(rng, mixed[::-1]),
            block(rng, mixed, controls=[ctl], cstates=[0])]


def run_blocks(q, n, dtype, gates, phi):
    st = q.State(n, dtype)
    if dtype == q.C128:
        st.set_arith(q.ARITH_F32X2)
    st.set_fused_tc(True)
    st.from_numpy(phi)
    for g in gates:
        st.apply_kq(g.matrix, g.qubits, g.controls, g.cstates)
    out = st.to_numpy().astype(np.complex128)
    st.free()
    return out


@pytest.mark.parametrize("n", [22, 24])
@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_multitile_blocks_against_oracle(q, n, k, dtype):
    dt = q.C128 if dtype == "c128" else q.C64
    tol = 1e-12 if dtype == "c128" else 2e-5
    rng = np.random.default_rng(1000 * n + 10 * k + dt)
    gates = placements(rng, n, k)
    phi = C.random_state(n, 50 + n)
    # amplitudes of O(1) in a few groups (an unnormalised vector, as in an adjoint co-state)
    phi[: 1 << 10] *= 30.0
    if dt == q.C64:
        phi = phi.astype(np.complex64).astype(np.complex128)   # the same input both sides
    ref = O.run_circuit(n, gates, phi)
    got = run_blocks(q, n, dt, gates, phi)
    err = np.abs(got - ref)
    assert float(err.max()) <= tol, (dtype, n, k, float(err.max()), int(err.argmax()))
    assert q.device_status()["tc_timeouts"] == 0


@pytest.mark.parametrize("dtype,mode", [("c64", 1), ("c64", 3), ("c128", 3), ("c128", 4)])
def test_wait_limit_reports_timeout_and_recovers(q, dtype, mode):
    dt = q.C128 if dtype == "c128" else q.C64
    n, k = 20, 5
    rng = np.random.default_rng(77 + dt)
    g = block(rng, [3, 7, 9, 12, 15])
    phi = C.random_state(n, 78)
    st = q.State(n, dt)
    if dt == q.C128:
        st.set_arith(q.ARITH_F32X2)
    st.set_fused_tc(mode)
    st.from_numpy(phi)
    st.set_wait_limit(-1)                      # every first MMA wait gives up at once
    st.apply_kq(g.matrix, g.qubits)
    with pytest.raises(q.QCError) as e:
        st.synchronize()
    assert e.value.code == q.QC_ERR_TIMEOUT
    st.synchronize()                           # reported once, then cleared
    assert q.device_status()["tc_timeouts"] == 0
    st.set_wait_limit(0)                       # default limit: the same block completes
    st.from_numpy(phi)
    st.apply_kq(g.matrix, g.qubits)
    got = st.to_numpy().astype(np.complex128)
    st.free()
    if dt == q.C64:
        phi = phi.astype(np.complex64).astype(np.complex128)
    ref = O.run_circuit(n, [g], phi)
    assert float(np.abs(got - ref).max()) <= (1e-12 if dt == q.C128 else 2e-5)


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("k", [3, 4, 5])
def test_kernel_variants_equal_register_loads(q, k, mode):
    """complex128 blocks: the one-role kernel with per-thread loads
    (qc_set_fused_tc 4), the same with tiles staged by the Tensor Memory
    Accelerator (2), the warp-specialised pipeline (3) and the default
    choice between them (1) run the same arithmetic, so the states agree bit
    for bit; all match the oracle.
    Placements: low, high and spread targets (TMA-staged in mode 2), and a
    control below the run length (per-thread loads in mode 2).  At n = 22 a
    CTA of the pipeline runs up to 2^15 / 152 tiles, so its A-buffer,
    accumulator-slot and row-scale rings all wrap many times."""
    n = 22
    rng = np.random.default_rng(500 + k)
    gates = placements(rng, n, k)
    phi = C.random_state(n, 501)
    phi[: 1 << 10] *= 30.0
    outs = []
    for mode in (4, mode):
        st = q.State(n, q.C128)
        st.set_arith(q.ARITH_F32X2)
        st.set_fused_tc(mode)
        st.from_numpy(phi)
        for g in gates:
            st.apply_kq(g.matrix, g.qubits, g.controls, g.cstates)
        outs.append(st.to_numpy())
        st.free()
    np.testing.assert_array_equal(outs[0], outs[1])
    ref = O.run_circuit(n, gates, phi)
    assert float(np.abs(outs[0] - ref).max()) <= 1e-12
    assert q.device_status()["tc_timeouts"] == 0


@pytest.mark.parametrize("k", [3, 4, 5])
def test_c64_pipeline_equals_one_role_kernel(q, k):
    """complex64 blocks: the warp-specialised pipeline (qc_set_fused_tc 3)
    computes the same split-TF32 products into the same accumulators as the
    one-role kernel (4), so the states agree bit for bit; both match the
    oracle.  n = 22: every CTA runs many tiles, so the A-buffer and
    accumulator-slot rings wrap many times."""
    n = 22
    rng = np.random.default_rng(700 + k)
    gates = placements(rng, n, k)
    phi = C.random_state(n, 701).astype(np.complex64)
    outs = []
    for mode in (4, 3):
        st = q.State(n, q.C64)
        st.set_fused_tc(mode)
        st.from_numpy(phi)
        for g in gates:
            st.apply_kq(g.matrix, g.qubits, g.controls, g.cstates)
        outs.append(st.to_numpy())
        st.free()
    np.testing.assert_array_equal(outs[0], outs[1])
    ref = O.run_circuit(n, gates, phi.astype(np.complex128))
    assert float(np.abs(outs[1].astype(np.complex128) - ref).max()) <= 2e-5
    assert q.device_status()["tc_timeouts"] == 0
