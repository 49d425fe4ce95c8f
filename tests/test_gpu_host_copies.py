"""GPU tests of the state's host copies.

qc_state_copy_from_host copies from page-locked host memory that CUDA has
mapped (here qcgb300.HostBuffer: cudaHostRegister) with a kernel reading that
memory, and from pageable memory with the copy engine; qc_state_copy_to_host
uses the copy engine.  Both directions must move every byte unchanged, for
both element types, from the smallest state (n = 1: 16 bytes in complex64)
up, and the mapped path must be ordered on the state's stream after the work
queued before it.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 5, 20])
def test_round_trip_through_mapped_and_pageable_memory(q, dtype, n):
    dt = q.C128 if dtype == "c128" else q.C64
    npdt = np.complex128 if dt == q.C128 else np.complex64
    rng = np.random.default_rng(10 * n + dt)
    src = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)).astype(npdt)
    st = q.State(n, dt)
    hb = q.HostBuffer(1 << n, dtype=npdt)
    try:
        hb.array[:] = src
        st.from_numpy(hb.array)                  # mapped page-locked memory
        got = st.to_numpy()
        assert got.tobytes() == src.tobytes()
        st.set_basis(0)
        st.from_numpy(src.copy())                # pageable memory
        got2 = st.to_numpy()
        assert got2.tobytes() == src.tobytes()
    finally:
        hb.free()
        st.free()


def test_mapped_copy_is_ordered_after_queued_work(q):
    """A gate queued before the copy from mapped memory must not touch the
    copied amplitudes: the copy overwrites its result, whatever the timing."""
    n = 22
    st = q.State(n, q.C128)
    hb = q.HostBuffer(1 << n)
    try:
        phi = C.random_state(n, 5)
        hb.array[:] = phi
        st.set_basis(0)
        st.apply_circuit(C.brickwork(n, 6, seed=2))   # queued work on the state's stream
        st.from_numpy(hb.array)
        got = st.to_numpy()
        assert got.tobytes() == phi.astype(np.complex128).tobytes()
    finally:
        hb.free()
        st.free()
