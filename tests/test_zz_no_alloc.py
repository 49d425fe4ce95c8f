"""qc_expect_noalloc through the C ABI against qc_expect.

qc_expect_noalloc serves callers that cannot allocate device memory (their
memory manager already holds the device, or a cudaMalloc would synchronise a
latency-critical loop): it keeps its partial sums in a fixed array in the
library's device code.  This test calls it twice in a row on the same states
-- the second call reuses the array as the first left it -- and checks both
results against the allocating entry point, within the expectation-value
tolerances of the other GPU tests, and against the FP64 oracle's value for
the same circuit.  It also checks that a sum needing more sweeps than the
fixed array holds is rejected without running.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_00123_gb300 import circuits as C

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


def call_noalloc(q, st, H):
    rec, keep = q.pauli_record(H)
    out = ctypes.c_double(float("nan"))
    rc = q.lib.qc_expect_noalloc(st.handle, ctypes.byref(rec), ctypes.byref(out))
    del keep
    return rc, out.value


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-12)])
def test_noalloc_matches_allocating_expect_twice(q, dtype, tol):
    n = 12
    st = q.State(n, q.C128 if dtype == "c128" else q.C64)
    gates = C.random_mix(n, 120, seed=44)
    st.apply_circuit(gates)
    psi = O.run_circuit(n, gates)
    H1 = C.tfim(n, 0.9) + [(0.3, [("Y", 1), ("X", 3)]), (-0.2, [("Y", 0), ("Z", 2), ("Y", 11)]), (0.5, [])]
    H2 = [(1.0, [("Z", i)]) for i in range(n)] + [(0.25, [("X", i), ("X", (i + 1) % n)]) for i in range(n)]
    for H in (H1, H2):
        ref = st.expect(H)
        rc1, v1 = call_noalloc(q, st, H)
        rc2, v2 = call_noalloc(q, st, H)
        assert rc1 == q.QC_OK and rc2 == q.QC_OK
        # both sum exact products of the same amplitudes with FP64-level accuracy (complex64: * sum|c|)
        t = tol * (1.0 if dtype == "c128" else max(1.0, sum(abs(c) for c, _ in H)))
        assert abs(v1 - ref) <= t and abs(v2 - ref) <= t
        # against the oracle: complex128 1e-10, complex64 state with FP64 reductions 2e-4
        assert abs(v1 - O.expect(psi, n, H)) <= (1e-10 if dtype == "c128" else 2e-4)
    st.free()


def test_noalloc_rejects_sums_beyond_its_limit(q):
    n = 12
    st = q.State(n, q.C128)
    # 1024 distinct X patterns need 1024 sweeps; the fixed scratch holds 1023
    H = [(1.0, [("X", b) for b in range(n) if (m >> b) & 1]) for m in range(1, 1025)]
    rc, _ = call_noalloc(q, st, H)
    assert rc == q.QC_ERR_ARG
    assert b"at most 1023" in q.lib.qc_last_error()
    rc, v = call_noalloc(q, st, [(2.0, [])])      # still usable afterwards
    assert rc == q.QC_OK and abs(v - 2.0) <= 1e-12
    st.free()
