"""Thin ctypes binding of the C ABI declared in ``include/qcgb300.h``.

Only argument marshalling lives here; every step of a gate sweep runs in the
CUDA kernels of ``libqcgb300.so``.  PyTorch is used for device memory and
streams (``State.from_tensor`` borrows a tensor's storage).  There is no CPU
fallback: importing this module fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqcgb300.so")

QC_OK, QC_ERR_ARG, QC_ERR_OOM, QC_ERR_CUDA, QC_ERR_TIMEOUT, QC_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
C64, C128 = 0, 1
ARITH_AUTO, ARITH_NATIVE, ARITH_F32X2 = 0, 1, 2
MAX_TARGETS, MAX_CONTROLS = 5, 8

GATE_KIND = {"MATRIX": 0, "U": 0, "U4": 0, "UK": 0, "H": 1, "X": 2, "Y": 3, "Z": 4, "S": 5, "SDG": 6,
             "T": 7, "TDG": 8, "P": 9, "RX": 10, "RY": 11, "RZ": 12, "SWAP": 13}


class QCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("qcgb300 error %d: %s" % (code, msg))
        self.code = code


class qc_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nq", ctypes.c_int), ("nc", ctypes.c_int),
                ("qubits", ctypes.c_int * MAX_TARGETS), ("controls", ctypes.c_int * MAX_CONTROLS),
                ("cstates", ctypes.c_int * MAX_CONTROLS), ("theta", ctypes.c_double),
                ("matrix", ctypes.POINTER(ctypes.c_double))]


class qc_opts(ctypes.Structure):
    _fields_ = [("fuse_k", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("gate_ms", ctypes.POINTER(ctypes.c_float)), ("nlaunch", ctypes.POINTER(ctypes.c_int))]


MAX_LIN = 36


class qc_block(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("qubits", ctypes.c_int * MAX_TARGETS), ("nc", ctypes.c_int),
                ("controls", ctypes.c_int * MAX_CONTROLS), ("cstates", ctypes.c_int * MAX_CONTROLS),
                ("U", ctypes.c_double * (2 * 32 * 32)), ("kind", ctypes.c_int), ("anchor", ctypes.c_int),
                ("nlin", ctypes.c_int), ("lin_qubits", ctypes.c_int * MAX_LIN),
                ("lin_theta", ctypes.c_double * MAX_LIN), ("theta0", ctypes.c_double)]


class qc_circuit_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("ngates", ctypes.c_int), ("gates", ctypes.POINTER(qc_gate))]


class qc_batch_opts(ctypes.Structure):
    _fields_ = [("fuse_k", ctypes.c_int), ("use_graph", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("spin_limit", ctypes.c_longlong), ("test_skip_circuit", ctypes.c_int),
                ("test_skip_member", ctypes.c_int)]


class qc_grad_opts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("arith", ctypes.c_int), ("stream", ctypes.c_void_p)]


class qc_shard_step(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("gate", qc_gate), ("rank_mask", ctypes.c_uint32),
                ("rank_val", ctypes.c_uint32), ("rank_bit", ctypes.c_int), ("local_qubit", ctypes.c_int)]


SHARD_GATE, SHARD_EXCHANGE = 0, 1


class qc_pauli_sum(ctypes.Structure):
    _fields_ = [("nterms", ctypes.c_int), ("coeffs", ctypes.POINTER(ctypes.c_double)),
                ("offsets", ctypes.POINTER(ctypes.c_int)), ("letters", ctypes.c_char_p),
                ("qubits", ctypes.POINTER(ctypes.c_int))]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libqcgb300.so not found at %s: run `python -c 'import __graft_entry__ as g; "
                          "g.build()'` (needs nvcc for sm_103a)" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    IP = ctypes.POINTER(ctypes.c_int)
    DP = ctypes.POINTER(ctypes.c_double)
    sig = {
        "qc_state_alloc": [I, I, ctypes.POINTER(P)],
        "qc_state_wrap": [P, I, I, ctypes.POINTER(P)],
        "qc_state_free": [P],
        "qc_state_set_basis": [P, ctypes.c_uint64],
        "qc_state_copy_to_host": [P, P],
        "qc_state_copy_from_host": [P, P],
        "qc_state_info": [P, ctypes.POINTER(P), IP, IP],
        "qc_set_stream": [P, P],
        "qc_set_arith": [P, I],
        "qc_set_fused_tc": [P, I],
        "qc_set_packed": [P, I],
        "qc_device_status": [IP],
        "qc_synchronize": [P],
        "qc_set_wait_limit": [P, ctypes.c_longlong],
        "qc_apply_1q": [P, DP, I],
        "qc_apply_c1q": [P, DP, IP, IP, I, I],
        "qc_apply_2q": [P, DP, I, I],
        "qc_apply_kq": [P, DP, IP, I, IP, IP, I],
        "qc_apply_circuit": [P, ctypes.POINTER(qc_gate), I, ctypes.POINTER(qc_opts)],
        "qc_expect": [P, ctypes.POINTER(qc_pauli_sum), DP],
        "qc_expect_noalloc": [P, ctypes.POINTER(qc_pauli_sum), DP],
        "qc_expect_passes": [I, I, ctypes.POINTER(qc_pauli_sum), IP],
        "qc_qasm_parse": [ctypes.c_char_p, ctypes.POINTER(P)],
        "qc_program_info": [P, IP, IP, IP],
        "qc_program_free": [P],
        "qc_qasm_write": [I, ctypes.POINTER(qc_gate), I, ctypes.c_char_p, ctypes.c_size_t,
                          ctypes.POINTER(ctypes.c_size_t)],
        "qc_fuse_plan": [I, ctypes.POINTER(qc_gate), I, I, ctypes.POINTER(qc_block), I, IP],
        "qc_adjoint_grad": [I, ctypes.POINTER(qc_gate), I, DP, I, ctypes.POINTER(qc_pauli_sum), DP, DP,
                            ctypes.POINTER(qc_grad_opts)],
        "qc_count_params": [ctypes.POINTER(qc_gate), I, IP],
        "qc_batch_create": [ctypes.POINTER(P), ctypes.POINTER(qc_circuit_desc), I, ctypes.POINTER(qc_batch_opts),
                            ctypes.POINTER(P)],
        "qc_batch_launch": [P, DP, DP],
        "qc_batch_info": [P, IP, IP, IP],
        "qc_batch_free": [P],
        "qc_shard_plan": [I, I, ctypes.POINTER(qc_gate), I, ctypes.POINTER(qc_shard_step), I, IP],
        "qc_shard_exchange": [P, P, I, I],
        "qc_shard_pack": [P, I, I, P],
        "qc_shard_unpack": [P, I, I, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.qc_last_error.restype = ctypes.c_char_p
    lib.qc_last_error.argtypes = []
    lib.qc_version.restype = ctypes.c_char_p
    lib.qc_version.argtypes = []
    return lib


lib = _load()


def _check(rc):
    if rc != QC_OK:
        raise QCError(rc, lib.qc_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iarr(seq):
    seq = [int(v) for v in seq]
    return (ctypes.c_int * max(1, len(seq)))(*seq)


def _mat(U) -> np.ndarray:
    """Complex matrix -> contiguous float64 (re, im) pairs."""
    U = np.ascontiguousarray(np.asarray(U, dtype=np.complex128))
    return U.view(np.float64).reshape(-1).copy()


# ------------------------------------------------------------------ records
def gate_records(gates):
    """Convert gate objects (name, qubits, controls, cstates, theta, matrix)
    into a ctypes array of qc_gate; returns (array, keepalive)."""
    arr = (qc_gate * max(1, len(gates)))()
    keep = []
    for i, g in enumerate(gates):
        name = g.name.upper()
        if name not in GATE_KIND:
            raise QCError(QC_ERR_ARG, "unknown gate name %r" % g.name)
        r = arr[i]
        r.kind = GATE_KIND[name]
        r.nq = len(g.qubits)
        controls = tuple(getattr(g, "controls", ()) or ())
        cstates = tuple(getattr(g, "cstates", ()) or ()) or (1,) * len(controls)
        if r.nq > MAX_TARGETS or len(controls) > MAX_CONTROLS:
            raise QCError(QC_ERR_ARG, "gate %d too wide" % i)
        r.nc = len(controls)
        for j, q in enumerate(g.qubits):
            r.qubits[j] = int(q)
        for j, (c, s) in enumerate(zip(controls, cstates)):
            r.controls[j] = int(c)
            r.cstates[j] = int(s)
        r.theta = float(g.theta) if getattr(g, "theta", None) is not None else 0.0
        if r.kind == 0:
            m = _mat(g.matrix)
            keep.append(m)
            r.matrix = _dptr(m)
    return arr, keep


def pauli_record(hamiltonian):
    """[(coeff, [(letter, qubit), ...]), ...] -> (qc_pauli_sum, keepalive)."""
    coeffs = np.array([float(c) for c, _ in hamiltonian], dtype=np.float64)
    offsets, letters, qubits = [0], [], []
    for _, ops in hamiltonian:
        for letter, q in ops:
            letters.append(letter.upper())
            qubits.append(int(q))
        offsets.append(len(letters))
    offs = _iarr(offsets)
    qs = _iarr(qubits)
    lt = ctypes.create_string_buffer("".join(letters).encode(), max(1, len(letters)))
    rec = qc_pauli_sum(len(coeffs), _dptr(coeffs) if len(coeffs) else None, offs,
                       ctypes.cast(lt, ctypes.c_char_p), qs)
    return rec, (coeffs, offs, qs, lt)


# ------------------------------------------------------------------ host memory
class HostBuffer:
    """Page-locked host memory for state copies (qc_state_copy_to_host /
    _from_host): an anonymous mapping advised for transparent huge pages and
    registered with CUDA (cudaHostRegister).  Huge pages keep the number of
    address translations the copy engine needs small; on GB300 a 17 GB
    host-to-device copy from such a buffer ran at 210 GB/s also right after a
    long sequence of gate sweeps, while the same copy from small-page pinned
    memory dropped to 20-50 GB/s there.  `array` is a numpy view of `count`
    elements of `dtype`; call free() (or let the object go) to unregister."""

    def __init__(self, count: int, dtype=np.complex128):
        import mmap
        import torch
        self.nbytes = int(count) * np.dtype(dtype).itemsize
        self._mm = mmap.mmap(-1, max(self.nbytes, 1), flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        try:
            self._mm.madvise(mmap.MADV_HUGEPAGE)
        except (AttributeError, OSError):
            pass                                  # no transparent huge pages: still page-locked below
        self.array = np.frombuffer(self._mm, dtype=dtype, count=int(count))
        self.array[:] = 0                         # touch every page before registering
        self._ptr = self.array.ctypes.data
        err = torch.cuda.cudart().cudaHostRegister(self._ptr, self.nbytes, 0)
        if int(getattr(err, "value", err)) != 0:
            raise QCError(QC_ERR_CUDA, "cudaHostRegister failed: %s" % err)
        self._registered = True

    def huge_page_bytes(self) -> int:
        """Bytes of the buffer backed by transparent huge pages (Linux smaps)."""
        lo_addr, tot, inside = self._ptr, 0, False
        try:
            with open("/proc/self/smaps") as f:
                for ln in f:
                    parts = ln.split()
                    if parts and "-" in parts[0] and ":" not in parts[0]:
                        a, b = (int(x, 16) for x in parts[0].split("-"))
                        inside = a < lo_addr + self.nbytes and b > lo_addr
                    elif inside and parts and parts[0] == "AnonHugePages:":
                        tot += int(parts[1]) * 1024
        except OSError:
            return -1
        return tot

    def free(self):
        if getattr(self, "_registered", False):
            import torch
            torch.cuda.cudart().cudaHostUnregister(self._ptr)
            self._registered = False
            self.array = None
            try:
                self._mm.close()
            except BufferError:       # a view of the buffer is still alive: the mapping goes with it
                pass

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ------------------------------------------------------------------ state
class State:
    """A 2^n-amplitude state in device memory (library-owned or borrowed)."""

    def __init__(self, n: int, dtype: int = C128, handle=None, tensor=None):
        self.n = n
        self.dtype = dtype
        self._tensor = tensor
        if handle is None:
            h = ctypes.c_void_p()
            _check(lib.qc_state_alloc(n, dtype, ctypes.byref(h)))
            handle = h
        self._h = handle

    @classmethod
    def from_tensor(cls, t):
        """Borrow a contiguous torch.complex64/complex128 CUDA tensor of 2^n entries."""
        import torch
        if not t.is_cuda or not t.is_contiguous():
            raise QCError(QC_ERR_ARG, "tensor must be a contiguous CUDA tensor")
        dtype = {torch.complex64: C64, torch.complex128: C128}.get(t.dtype)
        if dtype is None:
            raise QCError(QC_ERR_ARG, "tensor dtype must be complex64 or complex128")
        n = int(t.numel()).bit_length() - 1
        if (1 << n) != t.numel():
            raise QCError(QC_ERR_ARG, "tensor size is not a power of two")
        h = ctypes.c_void_p()
        _check(lib.qc_state_wrap(ctypes.c_void_p(t.data_ptr()), n, dtype, ctypes.byref(h)))
        return cls(n, dtype, handle=h, tensor=t)

    def free(self):
        if self._h is not None:
            _check(lib.qc_state_free(self._h))
            self._h = None

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None:
                lib.qc_state_free(self._h)
                self._h = None
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def np_dtype(self):
        return np.complex64 if self.dtype == C64 else np.complex128

    def set_stream(self, stream):
        """Bind a torch.cuda.Stream (or a raw cudaStream_t int / None)."""
        raw = getattr(stream, "cuda_stream", stream)
        _check(lib.qc_set_stream(self._h, ctypes.c_void_p(raw or 0)))

    def set_arith(self, arith: int):
        _check(lib.qc_set_arith(self._h, arith))

    def set_fused_tc(self, enable):
        """k>=3 blocks on the tensor cores (True/1, default), on the tensor cores with
        complex128 tiles staged by the TMA unit (2), or on the CUDA cores (False/0)."""
        _check(lib.qc_set_fused_tc(self._h, int(enable)))

    def set_packed(self, enable):
        """complex128 float-float sweeps: scalar FP32 (0/False), packed FP32 pairs (1/True),
        packed with fixed-binade chains for dense 2-qubit gates (2, the default)."""
        _check(lib.qc_set_packed(self._h, int(enable)))

    def set_wait_limit(self, polls: int):
        """Tensor-core MMA wait limit in polls (0: default; < 0: no poll, for tests)."""
        _check(lib.qc_set_wait_limit(self._h, int(polls)))

    def synchronize(self):
        """Wait for the state's stream; raises QCError(QC_ERR_TIMEOUT) when a
        tensor-core wait on its device gave up since the last report."""
        _check(lib.qc_synchronize(self._h))

    def set_basis(self, x: int = 0):
        _check(lib.qc_state_set_basis(self._h, ctypes.c_uint64(x)))

    def to_numpy(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(1 << self.n, dtype=self.np_dtype)
        _check(lib.qc_state_copy_to_host(self._h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def from_numpy(self, a):
        a = np.ascontiguousarray(a, dtype=self.np_dtype)
        assert a.size == (1 << self.n)
        _check(lib.qc_state_copy_from_host(self._h, ctypes.c_void_p(a.ctypes.data)))
        self._host_keep = a

    def device_ptr(self) -> int:
        p = ctypes.c_void_p()
        _check(lib.qc_state_info(self._h, ctypes.byref(p), None, None))
        return p.value

    # gates ---------------------------------------------------------------
    def apply_1q(self, U, target: int):
        m = _mat(U)
        _check(lib.qc_apply_1q(self._h, _dptr(m), int(target)))

    def apply_c1q(self, U, controls, cstates, target: int):
        m = _mat(U)
        _check(lib.qc_apply_c1q(self._h, _dptr(m), _iarr(controls), _iarr(cstates), len(controls), int(target)))

    def apply_2q(self, U4, q0: int, q1: int):
        m = _mat(U4)
        _check(lib.qc_apply_2q(self._h, _dptr(m), int(q0), int(q1)))

    def apply_kq(self, U, qubits, controls=(), cstates=()):
        m = _mat(U)
        _check(lib.qc_apply_kq(self._h, _dptr(m), _iarr(qubits), len(qubits), _iarr(controls),
                               _iarr(cstates or [1] * len(controls)), len(controls)))

    def apply_circuit(self, gates, fuse_k: int = 0, use_graph: bool = False, time_gates: bool = False):
        """Apply the gate list; returns (n_launches, per-launch ms or None)."""
        arr, keep = gate_records(gates)
        nl = ctypes.c_int(0)
        ms = (ctypes.c_float * max(1, len(gates)))() if time_gates else None
        o = qc_opts(int(fuse_k), int(bool(use_graph)),
                    ctypes.cast(ms, ctypes.POINTER(ctypes.c_float)) if ms is not None else None,
                    ctypes.pointer(nl))
        _check(lib.qc_apply_circuit(self._h, arr, len(gates), ctypes.byref(o)))
        del keep
        return nl.value, (np.array(ms[:nl.value], dtype=np.float64) if ms is not None else None)

    def expect(self, hamiltonian) -> float:
        rec, keep = pauli_record(hamiltonian)
        out = ctypes.c_double(0.0)
        _check(lib.qc_expect(self._h, ctypes.byref(rec), ctypes.byref(out)))
        del keep
        return out.value

    def expect_noalloc(self, hamiltonian) -> float:
        """qc_expect_noalloc: same value, no device allocation (fixed scratch)."""
        rec, keep = pauli_record(hamiltonian)
        out = ctypes.c_double(0.0)
        _check(lib.qc_expect_noalloc(self._h, ctypes.byref(rec), ctypes.byref(out)))
        del keep
        return out.value


def expect_passes(n: int, dtype: int, hamiltonian) -> int:
    """Host-only: how many passes over the state qc_expect makes for H."""
    rec, keep = pauli_record(hamiltonian)
    out = ctypes.c_int(0)
    _check(lib.qc_expect_passes(n, dtype, ctypes.byref(rec), ctypes.byref(out)))
    del keep
    return out.value


_KIND_NAME = {1: "H", 2: "X", 3: "Y", 4: "Z", 5: "S", 6: "SDG", 7: "T", 8: "TDG", 9: "P", 10: "RX", 11: "RY",
              12: "RZ", 13: "SWAP"}


def qasm_parse(text: str):
    """OpenQASM 2.0 text -> (nqubits, [Gate, ...], skipped measure/barrier count)."""
    from .circuits import Gate
    prog = ctypes.c_void_p()
    _check(lib.qc_qasm_parse(text.encode(), ctypes.byref(prog)))
    try:
        n, ng, ni = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(lib.qc_program_info(prog, ctypes.byref(n), ctypes.byref(ng), ctypes.byref(ni)))
        fn = lib.qc_program_gates
        fn.restype = ctypes.POINTER(qc_gate)
        fn.argtypes = [ctypes.c_void_p]
        recs = fn(prog)
        gates = []
        for i in range(ng.value):
            r = recs[i]
            qubits = tuple(r.qubits[:r.nq])
            controls = tuple(r.controls[:r.nc])
            cstates = tuple(r.cstates[:r.nc])
            if r.kind == 0:
                d = 1 << r.nq
                m = np.array([complex(r.matrix[2 * j], r.matrix[2 * j + 1]) for j in range(d * d)]).reshape(d, d)
                name = "U" if r.nq == 1 else ("U4" if r.nq == 2 else "UK")
                gates.append(Gate(name, qubits, controls=controls, cstates=cstates, matrix=m))
            else:
                gates.append(Gate(_KIND_NAME[r.kind], qubits, controls=controls, cstates=cstates,
                                  theta=float(r.theta)))
        return n.value, gates, ni.value
    finally:
        lib.qc_program_free(prog)


def qasm_write(n: int, gates) -> str:
    """Gate list -> OpenQASM 2.0 text over q[n]."""
    arr, keep = gate_records(gates)
    ln = ctypes.c_size_t(0)
    _check(lib.qc_qasm_write(n, arr, len(gates), None, 0, ctypes.byref(ln)))
    buf = ctypes.create_string_buffer(ln.value + 1)
    _check(lib.qc_qasm_write(n, arr, len(gates), buf, ln.value + 1, ctypes.byref(ln)))
    del keep
    return buf.value.decode()


def fuse_plan(n: int, gates, fuse_k: int):
    """Host-only launch plan: a list with one entry per launch, either a
    matrix block (qubits, controls, cstates, U) or a linear phase run
    ("phase", anchor, [(qubit, theta), ...], theta0, pre), where pre is None or
    a 2x2 matrix applied to the anchor first, in the same sweep, or a run of
    SWAPs on disjoint pairs applied as one bit permutation ("swap", [(a, b), ...])."""
    arr, keep = gate_records(gates)
    nb = ctypes.c_int(0)
    cap = max(1, len(gates))
    blocks = (qc_block * cap)()
    _check(lib.qc_fuse_plan(n, arr, len(gates), int(fuse_k), blocks, cap, ctypes.byref(nb)))
    out = []
    for b in blocks[:nb.value]:
        if b.kind == 2:
            out.append(("swap", [(b.lin_qubits[2 * j], b.lin_qubits[2 * j + 1]) for j in range(b.nlin // 2)]))
            continue
        if b.kind == 1:
            pre = None
            if b.k == 1:      # 2x2 matrix on the anchor, applied before the phase
                pre = np.array([complex(b.U[2 * i], b.U[2 * i + 1]) for i in range(4)]).reshape(2, 2)
            out.append(("phase", b.anchor, [(b.lin_qubits[j], b.lin_theta[j]) for j in range(b.nlin)], b.theta0,
                        pre))
            continue
        d = 1 << b.k
        U = np.array(b.U[:2 * d * d], dtype=np.float64).view(np.complex128).reshape(d, d)
        out.append((tuple(b.qubits[:b.k]), tuple(b.controls[:b.nc]), tuple(b.cstates[:b.nc]), U.copy()))
    del keep
    return out


def shard_plan(n: int, g: int, gates):
    """Steps that apply `gates` to an n-qubit state split over 2^g shards
    (qc_shard_plan).  Each step is ("gate", Gate, rank_mask, rank_val) -- the
    gate in shard qubit numbering, applied on ranks r with r & mask == val --
    or ("exchange", rank_bit, local_qubit)."""
    from .circuits import Gate
    arr, keep = gate_records(gates)
    ns = ctypes.c_int(0)
    _check(lib.qc_shard_plan(n, g, arr, len(gates), None, 0, ctypes.byref(ns)))
    steps = (qc_shard_step * max(1, ns.value))()
    _check(lib.qc_shard_plan(n, g, arr, len(gates), steps, ns.value, ctypes.byref(ns)))
    out = []
    for st in steps[:ns.value]:
        if st.kind == SHARD_EXCHANGE:
            out.append(("exchange", st.rank_bit, st.local_qubit))
            continue
        r = st.gate
        qubits = tuple(r.qubits[:r.nq])
        controls = tuple(r.controls[:r.nc])
        cstates = tuple(r.cstates[:r.nc])
        if r.kind == 0:
            d = 1 << r.nq
            m = np.array([complex(r.matrix[2 * j], r.matrix[2 * j + 1]) for j in range(d * d)]).reshape(d, d)
            name = "U" if r.nq == 1 else ("U4" if r.nq == 2 else "UK")
            gt = Gate(name, qubits, controls=controls, cstates=cstates, matrix=m)
        else:
            gt = Gate(_KIND_NAME[r.kind], qubits, controls=controls, cstates=cstates, theta=float(r.theta))
        out.append(("gate", gt, st.rank_mask, st.rank_val))
    del keep
    return out


def shard_exchange(a: "State", b: "State", local_qubit: int, bit_a: int):
    """Trade a's half {bit(local_qubit) = 1 - bit_a} with b's half {= bit_a} (one kernel)."""
    _check(lib.qc_shard_exchange(a.handle, b.handle, int(local_qubit), int(bit_a)))


def shard_pack(s: "State", local_qubit: int, bit: int, dev_ptr: int):
    _check(lib.qc_shard_pack(s.handle, int(local_qubit), int(bit), ctypes.c_void_p(dev_ptr)))


def shard_unpack(s: "State", local_qubit: int, bit: int, dev_ptr: int):
    _check(lib.qc_shard_unpack(s.handle, int(local_qubit), int(bit), ctypes.c_void_p(dev_ptr)))


def device_status() -> dict:
    t = ctypes.c_int(0)
    _check(lib.qc_device_status(ctypes.byref(t)))
    return {"tc_timeouts": t.value}


def count_params(gates) -> int:
    arr, keep = gate_records(gates)
    c = ctypes.c_int(0)
    _check(lib.qc_count_params(arr, len(gates), ctypes.byref(c)))
    return c.value


def adjoint_grad(n: int, gates, hamiltonian, thetas=None, dtype: int = C128, arith: int = ARITH_AUTO,
                 stream=None):
    """Energies [B] and adjoint gradients [B, P] of the parametric gates
    (RX/RY/RZ without controls).  thetas: None (use the gates' own angles) or
    an array [B, P] of angles for the parametric gates in circuit order."""
    arr, keep = gate_records(gates)
    P = count_params(gates)
    if thetas is None:
        B = 1
        th = None
    else:
        th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(-1, P) if P else
                                  np.zeros((np.asarray(thetas).shape[0], 0)))
        B = th.shape[0]
    rec, hk = pauli_record(hamiltonian)
    e = np.zeros(B, dtype=np.float64)
    g = np.zeros((B, max(P, 1)), dtype=np.float64)
    raw = getattr(stream, "cuda_stream", stream)
    o = qc_grad_opts(int(dtype), int(arith), ctypes.c_void_p(raw or 0))
    _check(lib.qc_adjoint_grad(n, arr, len(gates), _dptr(th) if th is not None and th.size else None, B,
                               ctypes.byref(rec), _dptr(e), _dptr(g), ctypes.byref(o)))
    del keep, hk
    return e, g[:, :P]


class Batch:
    """Many independent circuits in one persistent launch (qc_batch_*).
    `states[i]` receives circuits[i] applied to |0...0> at every launch()."""

    def __init__(self, states, circuits, fuse_k: int = -1, use_graph: bool = False, stream=None,
                 spin_limit: int = 0, test_skip=None):
        if len(states) != len(circuits) or not states:
            raise QCError(QC_ERR_ARG, "states and circuits must be non-empty and of equal length")
        self.states = list(states)
        self._keep = []
        descs = (qc_circuit_desc * len(circuits))()
        for i, (st, gates) in enumerate(zip(states, circuits)):
            arr, keep = gate_records(gates)
            self._keep.append((arr, keep))
            descs[i].n = st.n
            descs[i].ngates = len(gates)
            descs[i].gates = arr
        hs = (ctypes.c_void_p * len(states))(*[st.handle.value for st in states])
        raw = getattr(stream, "cuda_stream", stream)
        skip_c, skip_m = (test_skip[0] + 1, test_skip[1]) if test_skip else (0, 0)
        o = qc_batch_opts(int(fuse_k), int(bool(use_graph)), ctypes.c_void_p(raw or 0), int(spin_limit),
                          int(skip_c), int(skip_m))
        h = ctypes.c_void_p()
        _check(lib.qc_batch_create(hs, descs, len(states), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._keep = None   # gate records are only read during qc_batch_create

    def launch(self, timing: bool = False):
        """Run; with timing=True returns (completion_ms per circuit, total_ms)."""
        if not timing:
            _check(lib.qc_batch_launch(self._h, None, None))
            return None
        comp = np.zeros(len(self.states), dtype=np.float64)
        tot = ctypes.c_double(0.0)
        _check(lib.qc_batch_launch(self._h, _dptr(comp), ctypes.byref(tot)))
        return comp, tot.value

    def info(self):
        k, nops, nsm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.qc_batch_info(self._h, ctypes.byref(k), ctypes.byref(nops), ctypes.byref(nsm)))
        return {"fuse_k": k.value, "ops": nops.value, "smem_circuits": nsm.value}

    def free(self):
        if getattr(self, "_h", None) is not None:
            lib.qc_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def version() -> str:
    return lib.qc_version().decode()
