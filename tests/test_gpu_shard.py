"""One state over 2^g shards on one GPU: every shard is its own library state
and exchanges run as the library's in-place shard kernel (qc_shard_exchange).
The gathered result is compared element by element with the FP64 oracle of
the unsharded circuit (Eq. (1) gate by gate) at the amplitude tolerances
(1e-12 complex128, 2e-5 complex64), gate by gate and with fusion in every
shard.  Pack and unpack (the two ends of an exchange between processes) are
checked against the half they must copy.
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


def circuit(n, seed):
    rng = np.random.default_rng(seed)
    gates = C.random_mix(n, 150, seed=seed) + C.qft(n)
    for _ in range(8):
        qs = [int(v) for v in rng.choice(n, size=3, replace=False)]
        gates.append(Gate("UK", tuple(qs), matrix=C.haar_unitary(rng, 8)))
    gates.append(Gate("UK", (0, 1, 2), matrix=C.haar_unitary(rng, 8)))     # all targets global for g >= 3
    return gates


@pytest.mark.parametrize("fuse_k", [0, 4])
@pytest.mark.parametrize("g", [2, 3])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_sharded_run_matches_oracle(q, dtype, g, fuse_k):
    from paper_2303_00123_gb300 import shard
    n = 20
    dt = q.C128 if dtype == "c128" else q.C64
    gates = circuit(n, 300 + g)
    psi0 = C.random_state(n, 301)
    if dt == q.C64:
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    nloc = n - g
    states = []
    for r in range(1 << g):
        st = q.State(nloc, dt)
        st.from_numpy(psi0[r << nloc:(r + 1) << nloc])
        states.append(st)
    steps = shard.plan(n, g, gates)
    assert any(s[0] == "exchange" for s in steps)
    shard.run_single_device(states, n, g, steps, fuse_k=fuse_k)
    got = np.concatenate([st.to_numpy().astype(np.complex128) for st in states])
    for st in states:
        st.free()
    ref = O.run_circuit(n, gates, psi0)
    assert float(np.abs(got - ref).max()) <= (1e-12 if dt == q.C128 else 2e-5)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_pack_unpack_copy_exactly_one_half(q, dtype):
    import torch
    dt = q.C128 if dtype == "c128" else q.C64
    tdt = torch.complex128 if dt == q.C128 else torch.complex64
    n = 14
    psi = C.random_state(n, 7).astype(np.complex128 if dt == q.C128 else np.complex64)
    for local in (0, 5, n - 2, n - 1):
        for bit in (0, 1):
            st = q.State(n, dt)
            st.from_numpy(psi)
            buf = torch.empty(1 << (n - 1), dtype=tdt, device="cuda")
            q.shard_pack(st, local, bit, buf.data_ptr())
            idx = [y for y in range(1 << n) if ((y >> (n - 1 - local)) & 1) == bit]
            np.testing.assert_array_equal(buf.cpu().numpy(), psi[idx])
            dst = q.State(n, dt)
            dst.from_numpy(np.zeros_like(psi))
            q.shard_unpack(dst, local, bit, buf.data_ptr())
            want = np.zeros_like(psi)
            want[idx] = psi[idx]
            np.testing.assert_array_equal(dst.to_numpy(), want)
            st.free()
            dst.free()
