"""Seeded synthetic circuit and Hamiltonian generators.

This module only builds inputs: lists of gate records (names, qubits, angles,
Haar-random matrices drawn from a seeded numpy PCG64 generator) and Pauli sums.
It holds none of the simulation arithmetic; both the CUDA path and the CPU
oracle read its records and turn names into matrices with their own code.

Conventions of the records (QCLAB++ Sec. 2, Definition 1): qubit 0 is the most
significant bit of a basis index; a multi-qubit gate's matrix index reads its
target qubits in the listed order, the first one being the most significant
bit.  Named gates: H, X, Y, Z, S, SDG, T, TDG, P(theta), RX/RY/RZ(theta)
(= exp(-i theta P / 2)), SWAP; explicit matrices: U (2x2), U4 (4x4), UK.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Gate:
    name: str
    qubits: tuple
    controls: tuple = ()
    cstates: tuple = ()
    theta: float | None = None
    matrix: np.ndarray | None = field(default=None, repr=False)

    def __post_init__(self):
        self.qubits = tuple(int(q) for q in self.qubits)
        self.controls = tuple(int(q) for q in self.controls)
        if not self.cstates:
            self.cstates = (1,) * len(self.controls)
        self.cstates = tuple(int(s) for s in self.cstates)


def haar_unitary(rng: np.random.Generator, d: int) -> np.ndarray:
    """Haar-distributed d x d unitary: QR of a complex Ginibre matrix with the
    phases of R's diagonal moved into Q (Mezzadri 2007)."""
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return np.ascontiguousarray(q * ph[None, :])


# ---------------------------------------------------------------- circuits
def qft(n: int) -> list:
    """QFT circuit of Fig. 1: H on qubit i, then CP(control=j+i-1, target=i,
    theta=-2 pi / 2^j) for j=2..n-i, and finally SWAP(i, n-1-i)."""
    gates = []
    for i in range(n):
        gates.append(Gate("H", (i,)))
        for j in range(2, n - i + 1):
            gates.append(Gate("P", (i,), controls=(j + i - 1,), cstates=(1,), theta=-2.0 * math.pi / (1 << j)))
    for i in range(n // 2):
        gates.append(Gate("SWAP", (i, n - i - 1)))
    return gates


def brickwork(n: int, depth: int, seed: int) -> list:
    """`depth` layers; each layer is a Haar U(2) on every qubit followed by
    CNOTs on neighbour pairs (2i -> 2i+1 on even layers, 2i+1 -> 2i+2 on odd)."""
    rng = np.random.default_rng(seed)
    gates = []
    for layer in range(depth):
        for q in range(n):
            gates.append(Gate("U", (q,), matrix=haar_unitary(rng, 2)))
        start = 0 if layer % 2 == 0 else 1
        for c in range(start, n - 1, 2):
            gates.append(Gate("X", (c + 1,), controls=(c,), cstates=(1,)))
    return gates


def tfxy_trotter(n: int, steps: int, seed: int) -> list:
    """Trotter time evolution of a nearest-neighbour TFXY chain, the second
    benchmark circuit of Sec. 4 (its figure shows two steps on four qubits).
    One step: RZ on every qubit; on each even pair (i, i+1), i even: CNOT(i ->
    i+1), RX on i and RZ on i+1, CNOT(i -> i+1); RZ on every qubit; the same
    block on each odd pair.  Each block equals exp(-i a/2 X_i X_{i+1})
    exp(-i b/2 Z_i Z_{i+1}) for its RX angle a and RZ angle b.  The paper
    prints no angles: every angle is drawn uniformly from (-pi, pi), seeded."""
    rng = np.random.default_rng(seed)
    ang = lambda: float(rng.uniform(-math.pi, math.pi))
    gates = []
    for _ in range(steps):
        for start in (0, 1):
            for q in range(n):
                gates.append(Gate("RZ", (q,), theta=ang()))
            for i in range(start, n - 1, 2):
                gates.append(Gate("X", (i + 1,), controls=(i,), cstates=(1,)))
                gates.append(Gate("RX", (i,), theta=ang()))
                gates.append(Gate("RZ", (i + 1,), theta=ang()))
                gates.append(Gate("X", (i + 1,), controls=(i,), cstates=(1,)))
    return gates


def random_mix(n: int, ngates: int, seed: int) -> list:
    """Seeded gate mix: 60% Haar U(2) on a uniform target; 20% singly
    controlled gates (half CNOT, half controlled Haar U(2), control state 0/1
    uniform); 20% Haar U(4) on a uniform pair of distinct qubits."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(ngates):
        r = rng.random()
        if r < 0.6 or n < 2:
            gates.append(Gate("U", (int(rng.integers(n)),), matrix=haar_unitary(rng, 2)))
        elif r < 0.8:
            c, t = (int(v) for v in rng.choice(n, size=2, replace=False))
            st = int(rng.integers(2))
            if rng.random() < 0.5:
                gates.append(Gate("X", (t,), controls=(c,), cstates=(st,)))
            else:
                gates.append(Gate("U", (t,), controls=(c,), cstates=(st,), matrix=haar_unitary(rng, 2)))
        else:
            a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
            gates.append(Gate("U4", (a, b), matrix=haar_unitary(rng, 4)))
    return gates


def hea(n: int, layers: int, thetas) -> list:
    """Hardware-efficient ansatz: per layer RY(theta) on every qubit, then
    RZ(theta) on every qubit, then the CNOT ladder i -> i+1 (i = 0..n-2).
    `thetas` supplies 2*n*layers angles in gate order."""
    thetas = list(thetas)
    assert len(thetas) == 2 * n * layers
    gates, k = [], 0
    for _ in range(layers):
        for name in ("RY", "RZ"):
            for q in range(n):
                gates.append(Gate(name, (q,), theta=float(thetas[k])))
                k += 1
        for q in range(n - 1):
            gates.append(Gate("X", (q + 1,), controls=(q,), cstates=(1,)))
    return gates


def hea_thetas(n: int, layers: int, seed: int, batch: int | None = None) -> np.ndarray:
    """theta ~ U(-pi, pi), seeded; shape (2*n*layers,) or (batch, 2*n*layers)."""
    rng = np.random.default_rng(seed)
    shape = (2 * n * layers,) if batch is None else (batch, 2 * n * layers)
    return rng.uniform(-math.pi, math.pi, size=shape)


def tfim(n: int, h: float = 1.0) -> list:
    """Transverse-field Ising chain, open boundary:
    H = - sum_i Z_i Z_{i+1} - h sum_i X_i, as [(coeff, [(letter, qubit), ...])]."""
    terms = [(-1.0, [("Z", i), ("Z", i + 1)]) for i in range(n - 1)]
    terms += [(-h, [("X", i)]) for i in range(n)]
    return terms


def batch_specs(count: int, seed: int, nmin: int = 10, nmax: int = 24,
                dmin: int = 50, dmax: int = 300) -> list:
    """(n, depth, seed) triples of a batch of independent random circuits with
    qubit counts uniform in [nmin, nmax] and depths uniform in [dmin, dmax]."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count)
    ds = rng.integers(dmin, dmax + 1, size=count)
    return [(int(a), int(b), seed * 100003 + i) for i, (a, b) in enumerate(zip(ns, ds))]


def random_state(n: int, seed: int) -> np.ndarray:
    """Seeded normalised complex Gaussian state."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)
