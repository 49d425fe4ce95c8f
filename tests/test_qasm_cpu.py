"""OpenQASM 2.0 input and output (host code, no GPU): the parser's gates are
checked by applying them with the FP64 oracle against gate lists built from
the OpenQASM 2.0 definitions, and written programs are read back.

Pins: U(t, f, l) equals e^{i(f+l)/2} Rz(f) Ry(t) Rz(l) (the definition
U := Rz(f) Ry(t) Rz(l) up to a global phase); a user gate written as
rz(a/2) y; cx x,y; rz(-a/2) y; cx x,y equals controlled RZ(a) exactly."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_00123_gb300 import circuits as C
from paper_2303_00123_gb300.circuits import Gate


@pytest.fixture(scope="module")
def q():
    from paper_2303_00123_gb300 import build
    build.build()
    from paper_2303_00123_gb300 import qcgb300
    return qcgb300


def states_equal(n, a, b, phi, up_to_phase=False):
    x, y = O.run_circuit(n, a, phi), O.run_circuit(n, b, phi)
    if up_to_phase:
        ov = np.vdot(x, y)
        return abs(abs(ov) - 1.0) < 1e-12 and np.max(np.abs(x * ov / abs(ov) - y)) < 1e-12
    return np.max(np.abs(x - y)) < 1e-12


def test_u3_follows_the_openqasm_definition(q):
    t, f, l = 0.7, -1.1, 2.3
    n, g, _ = q.qasm_parse("OPENQASM 2.0; qreg a[1]; U(%r,%r,%r) a[0];" % (t, f, l))
    U = g[0].matrix
    ref = np.exp(0.5j * (f + l)) * (O.gate_matrix(Gate("RZ", (0,), theta=f)) @ O.gate_matrix(Gate("RY", (0,), theta=t))
                                    @ O.gate_matrix(Gate("RZ", (0,), theta=l)))
    np.testing.assert_allclose(U, ref, atol=1e-14)


PROGRAM = """
OPENQASM 2.0;
include "qelib1.inc";
// two registers: a -> qubits 0, 1, 2; b -> qubits 3, 4
qreg a[3];
qreg b[2];
creg c[5];
gate myrz(theta) x, y { rz(theta/2) y; cx x, y; rz(-theta/2) y; cx x, y; }
gate pair(p, r) u, v { myrz(p * 2) u, v; h u; barrier u, v; ry(sqrt(r) - pi/4) v; }
h a;                         // broadcast over the register
cx a[0], b[1];
pair(0.3, 2.0) b[0], a[2];
cu1(-pi/3) a[1], b[0];
u2(0.1, -0.2) b[1];
sx a[0]; sxdg a[0]; t b[0]; tdg a[1]; s a[2]; sdg b[1];
crx(0.25) b[1], a[0]; cry(-1.5) a[0], b[0]; crz(2*pi/7) a[2], a[1];
ccx a[0], a[1], b[0]; cswap b[1], a[0], a[2]; swap a[1], b[1];
rzz(0.9) a[0], b[0]; rxx(-0.4) a[2], b[1];
cu3(0.3, 0.2, 0.1) a[1], a[2]; cu(0.3, 0.2, 0.1, 0.5) b[0], b[1];
cx b[0], a[2];
measure a -> c;
barrier a;
"""


def test_program_with_definitions_broadcast_and_skipped_statements(q):
    text = PROGRAM
    n, g, ignored = q.qasm_parse(text)
    assert n == 5 and ignored == 2
    u3 = lambda t, f, l, gp=0.0: np.exp(1j * gp) * np.array(
        [[math.cos(t / 2), -np.exp(1j * l) * math.sin(t / 2)],
         [np.exp(1j * f) * math.sin(t / 2), np.exp(1j * (f + l)) * math.cos(t / 2)]])
    sx = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]])
    rzz = lambda t: np.diag(np.exp(-0.5j * t * np.array([1, -1, -1, 1])))
    X2 = np.fliplr(np.eye(4))
    rxx = lambda t: math.cos(t / 2) * np.eye(4) - 1j * math.sin(t / 2) * X2
    ref = [Gate("H", (0,)), Gate("H", (1,)), Gate("H", (2,)), Gate("X", (4,), controls=(0,)),
           # pair(0.3, 2.0) b[0], a[2]: myrz(0.6) 3, 2 == crz(0.6); h 3; ry(sqrt(2) - pi/4) 2
           Gate("RZ", (2,), controls=(3,), theta=0.6), Gate("H", (3,)), Gate("RY", (2,), theta=math.sqrt(2.0) - math.pi / 4),
           Gate("P", (3,), controls=(1,), theta=-math.pi / 3), Gate("U", (4,), matrix=u3(math.pi / 2, 0.1, -0.2)),
           Gate("U", (0,), matrix=sx), Gate("U", (0,), matrix=sx.conj().T), Gate("T", (3,)), Gate("TDG", (1,)),
           Gate("S", (2,)), Gate("SDG", (4,)),
           Gate("RX", (0,), controls=(4,), theta=0.25), Gate("RY", (3,), controls=(0,), theta=-1.5),
           Gate("RZ", (1,), controls=(2,), theta=2 * math.pi / 7),
           Gate("X", (3,), controls=(0, 1)), Gate("SWAP", (0, 2), controls=(4,)), Gate("SWAP", (1, 4)),
           Gate("U4", (0, 3), matrix=rzz(0.9)), Gate("U4", (2, 4), matrix=rxx(-0.4)),
           Gate("U", (2,), controls=(1,), matrix=u3(0.3, 0.2, 0.1)),
           Gate("U", (4,), controls=(3,), matrix=u3(0.3, 0.2, 0.1, 0.5)),
           Gate("X", (2,), controls=(3,))]
    assert len(g) == len(ref) + 3           # myrz expands to 4 gates (crz in the reference)
    phi = C.random_state(5, 3)
    assert states_equal(5, g, ref, phi)


def test_user_gate_equals_controlled_rz(q):
    text = """OPENQASM 2.0; qreg r[2];
gate myrz(theta) x, y { rz(theta/2) y; cx x, y; rz(-theta/2) y; cx x, y; }
myrz(1.3) r[0], r[1];"""
    n, g, _ = q.qasm_parse(text)
    assert states_equal(2, g, [Gate("RZ", (1,), controls=(0,), theta=1.3)], C.random_state(2, 8))


def test_broadcast_pairs_registers(q):
    n, g, _ = q.qasm_parse("OPENQASM 2.0; qreg a[3]; qreg b[3]; cx a, b; x b[1]; h a;")
    assert n == 6
    assert [(x.name, x.qubits, tuple(x.controls)) for x in g] == \
        [("X", (3,), (0,)), ("X", (4,), (1,)), ("X", (5,), (2,)), ("X", (4,), ()),
         ("H", (0,), ()), ("H", (1,), ()), ("H", (2,), ())]


@pytest.mark.parametrize("text,code", [
    ("OPENQASM 2.0; qreg q[2]; foo q[0];", -1),
    ("OPENQASM 2.0; qreg q[2]; h q[2];", -1),
    ("OPENQASM 2.0; qreg q[2]; cx q[0];", -1),
    ("OPENQASM 2.0; qreg q[2]; cx q[0], q[0];", -1),
    ("OPENQASM 2.0; qreg q[2]; rx q[0];", -1),
    ("OPENQASM 2.0; qreg q[2]; h q[0]", -1),
    ("OPENQASM 2.0; qreg q[2]; h r[0];", -1),
    ("OPENQASM 2.0; qreg q[2]; qreg q[1];", -1),
    ("OPENQASM 2.0; qreg q[2]; rz(bogus) q[0];", -1),
    ("OPENQASM 2.0; qreg q[2]; qreg r[3]; cx q, r;", -1),
    ("OPENQASM 2.0; h q[0];", -1),
    ("OPENQASM 2.0; qreg q[2]; reset q[0];", -5),
    ("OPENQASM 2.0; qreg q[2]; creg c[2]; if (c == 1) x q[0];", -5),
    ("OPENQASM 2.0; qreg q[2]; opaque g a;", -5),
    ("OPENQASM 3.0; qubit[2] q;", -5),
    ("OPENQASM 2.0; qreg q[2]; gate g a { g a; } g q[0];", -1),       # recursion
])
def test_errors(q, text, code):
    with pytest.raises(q.QCError) as e:
        q.qasm_parse(text)
    assert e.value.code == code


def test_write_and_read_back(q):
    """Named and controlled gates (control states 0 and 1), P/RX/RY/RZ,
    SWAP, Toffoli and singly controlled matrices are written exactly; an
    uncontrolled matrix comes back equal up to its global phase; 2-qubit
    matrices and doubly controlled rotations have no form here."""
    rng = np.random.default_rng(5)
    n = 6
    gates = C.qft(n) + [Gate("X", (2,), controls=(0, 4)), Gate("SWAP", (1, 5), controls=(3,), cstates=(0,)),
                        Gate("U", (2,), controls=(5,), cstates=(0,), matrix=C.haar_unitary(rng, 2)),
                        Gate("U", (0,), controls=(3,), matrix=C.haar_unitary(rng, 2)),
                        Gate("RY", (4,), controls=(1,), cstates=(0,), theta=0.7), Gate("Y", (3,), controls=(2,)),
                        Gate("SDG", (1,)), Gate("TDG", (0,)), Gate("RX", (5,), theta=-2.2)]
    text = q.qasm_write(n, gates)
    m, back, _ = q.qasm_parse(text)
    assert m == n
    phi = C.random_state(n, 6)
    assert states_equal(n, back, gates, phi)
    u = [Gate("U", (3,), matrix=C.haar_unitary(rng, 2))]
    assert states_equal(n, q.qasm_parse(q.qasm_write(n, u))[1], u, phi, up_to_phase=True)
    for bad in ([Gate("U4", (0, 1), matrix=C.haar_unitary(rng, 4))], [Gate("RZ", (0,), controls=(1, 2), theta=0.1)]):
        with pytest.raises(q.QCError) as e:
            q.qasm_write(n, bad)
        assert e.value.code == q.QC_ERR_UNSUPPORTED
