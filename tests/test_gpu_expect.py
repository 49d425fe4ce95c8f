"""GPU parity for qc_expect (tiled passes) against the FP64 oracle.

qc_expect groups the Pauli terms into passes over tiles of 2^12 (complex128)
or 2^13 (complex64) amplitudes; the host chooses each pass's generator masks
so that every term's X/Y pattern lies in the span of one pass.  These cases
drive that planning through its branches -- small states held in one tile,
terms whose flip masks need more generators than one pass has, many terms
sharing a flip mask (more than the four evaluated together), diagonal-only
sums, Y-odd strings (Im w) -- and compare against oracle.expect.  At 28 and 30
qubits the reference is a closed form: on a product state every Pauli string
factorises into single-qubit Bloch components.

Tolerance: complex128 1e-12 absolute on sums of O(1) coefficients (the
float-float arithmetic carries 47-bit amplitudes and exact hi*hi products);
complex64 1e-12 * max(1, sum |c_t|) against the oracle evaluated on the same
(complex64) amplitudes: the FP32 amplitudes' products are exact in two floats
and every sum is a fixed-binade chain or float-float (about 2^-46 of
sum |c_t|), i.e. the reductions keep FP64-level accuracy.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_00123_gb300 import circuits as C
from paper_2303_00123_gb300.circuits import Gate

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-12}


def tol(dtype, H):
    return TOL[dtype] * (1.0 if dtype == "c128" else max(1.0, sum(abs(c) for c, _ in H)))


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00123_gb300 import build
    build.build()
    from paper_2303_00123_gb300 import qcgb300
    return qcgb300


def random_sum(n, nterms, seed, max_len=None, letters="XYZI"):
    rng = np.random.default_rng(seed)
    H = []
    for _ in range(nterms):
        k = int(rng.integers(0, (max_len or n) + 1))
        qs = rng.choice(n, size=min(k, n), replace=False)
        ops = [(letters[int(rng.integers(0, len(letters)))], int(qb)) for qb in qs]
        H.append((float(rng.uniform(-1, 1)), ops))
    return H


def check(q, n, dtype, H, seed=5):
    psi = C.random_state(n, seed)
    st = q.State(n, q.C128 if dtype == "c128" else q.C64)
    st.from_numpy(psi)
    ref_psi = st.to_numpy().astype(np.complex128)      # the amplitudes the device holds
    ref = O.expect(ref_psi, n, H)
    got = st.expect(H)
    st.free()
    assert abs(got - ref) <= tol(dtype, H), (n, dtype, got, ref)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 9, 12, 13, 14, 16])
def test_random_pauli_sums(q, dtype, n):
    H = random_sum(n, 40, seed=100 + n)
    H += [(0.7, []), (-0.4, [("Z", 0)]), (0.3, [("X", n - 1)]), (0.2, [("Y", n // 2)])]
    check(q, n, dtype, H, seed=n)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_full_length_strings_need_many_passes(q, dtype):
    """n=18: strings over all 18 qubits; their high X/Y patterns span far more
    than one pass's generators, so the planner opens several passes."""
    n = 18
    H = random_sum(n, 24, seed=7, max_len=n, letters="XY")
    H += random_sum(n, 8, seed=8, max_len=n, letters="XYZ")
    check(q, n, dtype, H)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_many_terms_share_a_flip_mask(q, dtype):
    """n=15: 11 terms with flip mask {X_3, X_12} and different Z/Y phase masks
    (split into groups of four), plus 37 diagonal terms."""
    n = 15
    rng = np.random.default_rng(21)
    H = []
    for i in range(11):
        zs = [("Z", int(b)) for b in rng.choice([b for b in range(n) if b not in (3, 12)], size=i % 5, replace=False)]
        a = "Y" if i % 3 == 0 else "X"
        H.append((float(rng.uniform(-1, 1)), [(a, 3), ("X", 12)] + zs))
    for i in range(37):
        qs = rng.choice(n, size=int(rng.integers(1, 6)), replace=False)
        H.append((float(rng.uniform(-1, 1)), [("Z", int(b)) for b in qs]))
    check(q, n, dtype, H)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_more_register_groups_than_staged(q, dtype):
    """n=13, one pass: every flip mask inside each 4-bit register window
    (index bits 4a .. 4a+3, a = 0, 1, 2), each with three groups -- X only
    plus the same X times Z on the global bit 12 (one unsigned group of two
    terms whose signs differ between the two tiles), X times Z on two tile
    bits outside the flip (one signed group of two terms), and a Y on the
    lowest flip bit (an Im-weighted signed group): 135 pair groups, more than
    the 128 whose records and weights a tile stages in shared memory."""
    n = 13
    qubit = lambda b: n - 1 - b            # qubit whose index bit is b
    rng = np.random.default_rng(33)
    H = []
    for a in range(3):
        for f in range(1, 16):
            bits = [4 * a + b for b in range(4) if (f >> b) & 1]
            xs = [("X", qubit(b)) for b in bits]
            free = [b for b in range(12) if b not in bits]
            z1, z2 = (int(b) for b in rng.choice(free, size=2, replace=False))
            c = rng.uniform(-1, 1, size=5)
            H.append((float(c[0]), xs))
            H.append((float(c[1]), xs + [("Z", qubit(12))]))
            H.append((float(c[2]), xs + [("Z", qubit(z1))]))
            H.append((float(c[3]), xs + [("Z", qubit(z2))]))
            H.append((float(c[4]), [("Y", qubit(bits[0]))] + xs[1:]))
    assert q.expect_passes(n, q.C128 if dtype == "c128" else q.C64, H) == 1
    check(q, n, dtype, H, seed=41)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_hamiltonian_families(q, dtype):
    n = 14
    heis = []
    for i in range(n - 1):
        for L in "XYZ":
            heis.append((0.5 + 0.1 * i, [(L, i), (L, i + 1)]))
    check(q, n, dtype, C.tfim(n, 0.7))
    check(q, n, dtype, heis)
    check(q, n, dtype, [(1.0, [])])
    check(q, n, dtype, [(0.25, [("Z", i)]) for i in range(n)])


def bloch(a, phi):
    return {"I": 1.0, "X": math.sin(2 * a) * math.cos(phi), "Y": math.sin(2 * a) * math.sin(phi),
            "Z": math.cos(2 * a)}


@pytest.mark.parametrize("dtype,n", [("c128", 28), ("c64", 30)])
def test_product_state_closed_form_full_size(q, dtype, n):
    """Product state prod_i (cos a_i |0> + e^{i phi_i} sin a_i |1>), prepared
    on the device by RY(2 a_i) and P(phi_i): every Pauli string's value is the
    product of single-qubit Bloch components sin2a cos phi, sin2a sin phi,
    cos2a -- at any size, independent of the oracle."""
    import torch
    rng = np.random.default_rng(90 + n)
    a = rng.uniform(0.05, 1.5, size=n)
    phi = rng.uniform(-math.pi, math.pi, size=n)
    gates = []
    for i in range(n):
        gates.append(Gate("RY", (i,), theta=float(2 * a[i])))
        gates.append(Gate("P", (i,), theta=float(phi[i])))
    H = C.tfim(n, 0.9) + random_sum(n, 30, seed=n, max_len=n) + [(0.5, [("X", i) for i in range(n)])]
    ref = 0.0
    for c, ops in H:
        v = c
        for L, qb in ops:
            v *= bloch(a[qb], phi[qb])[L.upper()]
        ref += v
    t = torch.zeros(1 << n, dtype=torch.complex128 if dtype == "c128" else torch.complex64, device="cuda")
    st = q.State.from_tensor(t)
    st.set_basis(0)
    st.apply_circuit(gates)
    got = st.expect(H)
    st.free()
    del t
    torch.cuda.empty_cache()
    # complex64: the state itself carries ~1e-7 relative rounding per gate
    assert abs(got - ref) <= (1e-11 if dtype == "c128" else 2e-4 * sum(abs(c) for c, _ in H))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_repeated_and_reordered_terms(q, dtype):
    """Terms with equal flip and phase masks are combined on the host: the
    same string listed twice, written in another qubit order, or cancelling."""
    n = 13
    H = [(0.3, [("X", 2), ("Y", 7)]), (0.2, [("Y", 7), ("X", 2)]), (-0.5, [("X", 2), ("Y", 7)]),
         (0.7, [("Z", 1), ("X", 9), ("Z", 12)]), (0.7, [("Z", 12), ("X", 9), ("Z", 1)]),
         (1.1, [("Y", 0), ("Y", 12)]), (-1.1, [("Y", 12), ("Y", 0)]), (0.4, [("Z", 5)]), (0.4, [("Z", 5)])]
    check(q, n, dtype, H, seed=77)


def test_qft_state_closed_form_n30(q):
    """n=30 complex128, the QFT of a basis state |x> (a product state):
    |psi_y|^2 = 1/N makes every ZZ term vanish and <X_q> = cos(2 pi x 2^b / N),
    b = n-1-q, so the TFIM energy is -sum_q cos(2 pi x 2^b / N) -- a reference
    at full size independent of the oracle, sensitive to how the 2^30-term
    reduction accumulates."""
    import torch
    n = 30
    x = 123456789 % (1 << n)
    t = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    st = q.State.from_tensor(t)
    st.set_basis(x)
    st.apply_circuit(C.qft(n), fuse_k=2)
    ref = -sum(math.cos(2 * math.pi * ((x << (n - 1 - qq)) % (1 << n)) / (1 << n)) for qq in range(n))
    got = st.expect(C.tfim(n, 1.0))
    st.free()
    del t
    torch.cuda.empty_cache()
    assert abs(got - ref) <= 1e-12 * n
