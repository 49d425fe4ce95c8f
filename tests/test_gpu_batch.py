"""GPU parity of the batched persistent launch (qc_batch_*) against the FP64
oracle, circuit by circuit."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_00123_gb300 import circuits as C

pytestmark = pytest.mark.gpu
TOL = {"c128": 1e-12, "c128x": 1e-12, "c64": 2e-5}


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00123_gb300 import build
    build.build()
    from paper_2303_00123_gb300 import qcgb300
    return qcgb300


def make_states(q, ns, mode):
    sts = []
    for n in ns:
        st = q.State(n, q.C64 if mode == "c64" else q.C128)
        if mode == "c128":
            st.set_arith(q.ARITH_NATIVE)
        elif mode == "c128x":
            st.set_arith(q.ARITH_F32X2)
        sts.append(st)
    return sts


@pytest.mark.parametrize("mode", ["c64", "c128x", "c128"])
@pytest.mark.parametrize("fuse_k", [0, 2, 4, -1])
def test_batch_matches_oracle(q, mode, fuse_k):
    """Mixed sizes (shared-memory and global-memory circuits) and depths."""
    specs = C.batch_specs(24, seed=5, nmin=2, nmax=15, dmin=5, dmax=60)
    circs = [C.random_mix(n, d, seed=s) for n, d, s in specs]
    sts = make_states(q, [n for n, _, _ in specs], mode)
    for st in sts:                      # garbage in the states: the batch must start from |0>
        st.set_basis((1 << st.n) - 1)
    b = q.Batch(sts, circs, fuse_k=fuse_k)
    comp, tot = b.launch(timing=True)
    assert np.all(comp > 0) and np.all(comp <= tot * 1.01 + 0.05)
    for (n, d, s), st, g in zip(specs, sts, circs):
        got = st.to_numpy().astype(np.complex128)
        assert np.max(np.abs(got - O.run_circuit(n, g))) <= TOL[mode], (n, d)
    info = b.info()
    assert info["smem_circuits"] > 0 and info["smem_circuits"] < len(specs)
    b.free()
    for st in sts:
        st.free()


def test_batch_graph_replay_and_wide_controls(q):
    import torch
    n_list = [4, 9, 14, 16]
    circs = []
    for i, n in enumerate(n_list):
        g = C.random_mix(n, 40, seed=70 + i)
        g.append(C.Gate("X", (0,), controls=tuple(range(1, min(n, 8))), cstates=tuple([1, 0] * 4)[:min(n, 8) - 1]))
        g += C.qft(n)
        circs.append(g)
    sts = make_states(q, n_list, "c64")
    s = torch.cuda.Stream()
    b = q.Batch(sts, circs, fuse_k=3, use_graph=True, stream=s)
    for rep in range(2):                # replays restart from |0...0>
        b.launch()
        s.synchronize()
        for n, st, g in zip(n_list, sts, circs):
            assert np.max(np.abs(st.to_numpy().astype(np.complex128) - O.run_circuit(n, g))) <= 2e-5
    b.free()


def test_batch_rejects_mismatched_states(q):
    sts = make_states(q, [5, 6], "c64")
    with pytest.raises(q.QCError):   # a gate on qubit 6 of a 6-qubit state
        q.Batch(sts, [C.random_mix(5, 3, seed=1), [C.Gate("H", (6,))]])
    st128 = q.State(6, q.C128)
    with pytest.raises(q.QCError):
        q.Batch([sts[0], st128], [C.random_mix(5, 3, seed=1), C.random_mix(6, 3, seed=2)])


def test_batch_full_config_sampled(q):
    """1024 circuits, n ~ U[10, 24], depth ~ U[50, 300], complex64, autotuned
    fusion, graph replay: final states of sampled circuits against the oracle."""
    import torch
    specs = C.batch_specs(1024, seed=4)
    circs = [C.random_mix(n, d, seed=s) for n, d, s in specs]
    sts = make_states(q, [n for n, _, _ in specs], "c64")
    s = torch.cuda.Stream()
    b = q.Batch(sts, circs, fuse_k=-1, use_graph=True, stream=s)
    comp, tot = b.launch(timing=True)
    assert len(comp) == 1024 and tot > 0
    idx = sorted(range(1024), key=lambda i: specs[i][0])
    sample = idx[:2] + idx[500:502] + [i for i in idx[::-1] if specs[i][0] <= 20][:1]
    for i in sample:
        n, d, _ = specs[i]
        got = sts[i].to_numpy().astype(np.complex128)
        assert np.max(np.abs(got - O.run_circuit(n, circs[i]))) <= 2e-5, (i, n, d)
    b.free()


def test_batch_teams_match_oracle(q):
    """States above 8 MB (complex64 n >= 21) are swept by CTA teams with
    barriers between gate blocks; results against the oracle."""
    specs = [(21, 30, 501), (22, 25, 502), (12, 40, 503), (23, 12, 504), (16, 30, 505)]
    circs = [C.random_mix(n, d, seed=s) for n, d, s in specs]
    sts = make_states(q, [n for n, _, _ in specs], "c64")
    b = q.Batch(sts, circs, fuse_k=3)
    comp, tot = b.launch(timing=True)
    for (n, d, s), st, g in zip(specs, sts, circs):
        assert np.max(np.abs(st.to_numpy().astype(np.complex128) - O.run_circuit(n, g))) <= 2e-5, n
    b.free()


def test_batch_barrier_timeout_is_reported(q):
    """A team member that never arrives (host-set test flag) makes the other
    members' bounded waits give up; the launch returns QC_ERR_TIMEOUT and the
    device stays usable."""
    specs = [(22, 10, 601), (10, 10, 602)]
    circs = [C.random_mix(n, d, seed=s) for n, d, s in specs]
    sts = make_states(q, [n for n, _, _ in specs], "c64")
    b = q.Batch(sts, circs, fuse_k=2, spin_limit=20000, test_skip=(0, 1))
    with pytest.raises(q.QCError) as ei:
        b.launch(timing=True)
    assert ei.value.code == q.QC_ERR_TIMEOUT
    b.free()
    b2 = q.Batch(sts, circs, fuse_k=2)                 # a normal launch afterwards works
    b2.launch(timing=True)
    for (n, d, s), st, g in zip(specs, sts, circs):
        assert np.max(np.abs(st.to_numpy().astype(np.complex128) - O.run_circuit(n, g))) <= 2e-5
    b2.free()
