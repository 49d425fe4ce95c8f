"""Plain FP64 CPU oracle for the QCLAB++ gate-simulation hot path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA implementation and never imports it.

Contents, each following the passage it cites:

* gate matrices for the named gates of the paper's circuits (QFT of Fig. 1:
  H, CP, SWAP; Trotter circuit of Fig. 5: Rz, Rx, CNOT) and the readings the
  paper leaves open (P(theta) = diag(1, e^{i theta}); R_P(theta) =
  exp(-i theta P / 2));
* gate application: ``qc_oracle.c`` walks every basis index and applies
  Eq. (1) group by group (Definition 1 bit order, q_0 = most significant bit
  of a multi-qubit gate's matrix index);
* expectation values of Pauli sums: each Pauli string is applied explicitly
  as single-qubit X/Y/Z gates and the inner product is taken in FP64;
* gradients of exp(-i theta P / 2) gates: the parameter-shift rule
  g = [E(theta + pi/2) - E(theta - pi/2)] / 2 (Mitarai et al. 2018, Schuld et
  al. 2019), and central finite differences.

Gates are duck-typed records with the attributes ``name``, ``qubits``,
``controls``, ``cstates``, ``theta`` and ``matrix``.
"""
from __future__ import annotations

import copy
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile qc_oracle.c with gcc (OpenMP, -O2) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fcx-limited-range",
                               "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            ip = ctypes.POINTER(ctypes.c_int)
            lib.orc_apply_gate.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ip, ctypes.c_int, ip, ip, ctypes.c_int]
            lib.orc_apply_gate.restype = ctypes.c_int
            _lib = lib
    return _lib


# --------------------------------------------------------------------------
# Gate matrices (row-major, complex128)
# --------------------------------------------------------------------------
_SQ2 = 1.0 / np.sqrt(2.0)
_FIXED = {
    "I": np.eye(2, dtype=np.complex128),
    "H": np.array([[_SQ2, _SQ2], [_SQ2, -_SQ2]], dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
    "S": np.array([[1, 0], [0, 1j]], dtype=np.complex128),
    "SDG": np.array([[1, 0], [0, -1j]], dtype=np.complex128),
    "T": np.array([[1, 0], [0, np.exp(1j * np.pi / 4)]], dtype=np.complex128),
    "TDG": np.array([[1, 0], [0, np.exp(-1j * np.pi / 4)]], dtype=np.complex128),
    # Sec. 2.3: SWAP exchanges |01> and |10>.
    "SWAP": np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128),
}


def gate_matrix(g) -> np.ndarray:
    """Matrix of the (uncontrolled part of the) gate ``g``."""
    name = g.name.upper()
    if name in _FIXED:
        return _FIXED[name]
    t = g.theta
    if name == "P":   # phase gate P(theta) = diag(1, e^{i theta})
        return np.array([[1, 0], [0, np.exp(1j * t)]], dtype=np.complex128)
    if name == "RX":  # exp(-i theta X / 2)
        c, s = np.cos(t / 2), np.sin(t / 2)
        return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)
    if name == "RY":  # exp(-i theta Y / 2)
        c, s = np.cos(t / 2), np.sin(t / 2)
        return np.array([[c, -s], [s, c]], dtype=np.complex128)
    if name == "RZ":  # exp(-i theta Z / 2)
        return np.array([[np.exp(-0.5j * t), 0], [0, np.exp(0.5j * t)]], dtype=np.complex128)
    if name in ("U", "U4", "UK"):
        return np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128))
    raise ValueError("oracle: unknown gate %r" % g.name)


# --------------------------------------------------------------------------
# State and gate application
# --------------------------------------------------------------------------
def basis_state(n: int, x: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[x] = 1.0
    return psi


def _ints(seq):
    seq = list(seq)
    arr = (ctypes.c_int * max(1, len(seq)))(*seq)
    return arr, len(seq)


def apply_matrix(psi: np.ndarray, n: int, U: np.ndarray, qubits, controls=(), cstates=None) -> None:
    """psi <- (controlled) U on `qubits`, in place (Eq. (1), Sec. 2.2-2.4)."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == (1 << n)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    k = len(qubits)
    assert U.shape == (1 << k, 1 << k)
    if cstates is None:
        cstates = [1] * len(controls)
    q, kq = _ints(qubits)
    c, nc = _ints(controls)
    s, _ = _ints(cstates)
    rc = _load().orc_apply_gate(n, psi.ctypes.data, U.ctypes.data, q, kq, c, s, nc)
    if rc != 0:
        raise ValueError("oracle: invalid gate qubits=%r controls=%r (n=%d)" % (qubits, controls, n))


def apply_gate(psi: np.ndarray, n: int, g) -> None:
    controls = tuple(getattr(g, "controls", ()) or ())
    cstates = getattr(g, "cstates", None)
    if cstates is None or len(cstates) == 0:
        cstates = (1,) * len(controls)
    apply_matrix(psi, n, gate_matrix(g), tuple(g.qubits), controls, cstates)


def run_circuit(n: int, gates, psi0: np.ndarray | None = None) -> np.ndarray:
    """Final state of `gates` applied in order to psi0 (default |0...0>)."""
    psi = basis_state(n, 0) if psi0 is None else np.array(psi0, dtype=np.complex128, copy=True)
    for g in gates:
        apply_gate(psi, n, g)
    return psi


# --------------------------------------------------------------------------
# Pauli sums and expectation values
# --------------------------------------------------------------------------
def apply_pauli_string(psi: np.ndarray, n: int, ops) -> np.ndarray:
    """Return P|psi> for the Pauli string `ops` = [(letter, qubit), ...]."""
    out = psi.copy()
    for letter, q in ops:
        letter = letter.upper()
        if letter == "I":
            continue
        apply_matrix(out, n, _FIXED[letter], (q,))
    return out


def expect(psi: np.ndarray, n: int, hamiltonian) -> float:
    """<psi| sum_t c_t P_t |psi> in FP64; `hamiltonian` = [(c_t, ops_t), ...]."""
    total = 0.0
    for coeff, ops in hamiltonian:
        total += coeff * np.vdot(psi, apply_pauli_string(psi, n, ops)).real
    return float(total)


def energy(n: int, gates, hamiltonian, psi0=None) -> float:
    return expect(run_circuit(n, gates, psi0), n, hamiltonian)


PARAMETRIC = ("RX", "RY", "RZ")


def parametric_indices(gates):
    """Indices of gates of the form exp(-i theta P / 2) (controls not allowed)."""
    return [i for i, g in enumerate(gates)
            if g.name.upper() in PARAMETRIC and not (getattr(g, "controls", ()) or ())]


def _with_theta(gates, i, theta):
    out = list(gates)
    g = copy.copy(out[i])
    g.theta = theta
    out[i] = g
    return out


def param_shift_grad(n: int, gates, hamiltonian, psi0=None) -> np.ndarray:
    """dE/dtheta for every exp(-i theta P/2) gate, by the parameter-shift rule."""
    idx = parametric_indices(gates)
    g = np.zeros(len(idx))
    for k, i in enumerate(idx):
        t = gates[i].theta
        ep = energy(n, _with_theta(gates, i, t + np.pi / 2), hamiltonian, psi0)
        em = energy(n, _with_theta(gates, i, t - np.pi / 2), hamiltonian, psi0)
        g[k] = 0.5 * (ep - em)
    return g


def finite_diff_grad(n: int, gates, hamiltonian, h: float = 1e-4, psi0=None) -> np.ndarray:
    """Central finite differences [E(theta+h) - E(theta-h)] / (2h)."""
    idx = parametric_indices(gates)
    g = np.zeros(len(idx))
    for k, i in enumerate(idx):
        t = gates[i].theta
        ep = energy(n, _with_theta(gates, i, t + h), hamiltonian, psi0)
        em = energy(n, _with_theta(gates, i, t - h), hamiltonian, psi0)
        g[k] = (ep - em) / (2 * h)
    return g
