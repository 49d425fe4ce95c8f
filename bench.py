"""Benchmark: gate throughput of the state-vector engine on GB300.

Workload (one step): the two n=30 complex128 circuits of the large-state
configuration, applied gate by gate through qc_apply_circuit from a seeded
basis state -- the QFT circuit of QCLAB++ Fig. 1 (480 gates: 30 H, 435
controlled phases, 15 SWAP) and a depth-40 brickwork circuit (1200 Haar U(2),
580 CNOT).  `value` = gates per second over both circuits (device time, inputs
resident in HBM; the 17.2 GB state is far larger than the 129 MB L2, so no
flush is needed between launches).

Extra keys: `roofline` of the dominant kernel (dense 1-qubit sweep) from the
per-launch CUDA-event times recorded on the launching stream; `e2e` through the
C ABI with pinned host buffers (host->device state copy, circuits, device->host
copy of the final state); `cpu_baseline` = the FP64 CPU oracle timed on a
bounded sample on this machine's host cores; `clocks` sampled with nvidia-smi
during the timed region.  `--impl reference` times the oracle alone.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2303_00123_gb300 import circuits as C  # noqa: E402

N_QUBITS = 30
BRICK_DEPTH = 40
SEED_BASIS = 1000
SEED_BRICK = 1001
TFXY_STEPS = 10          # TFXY Trotter circuit: 10 steps = 1760 gates at n=30
TFXY_C128_K = 5          # its fastest complex128 fusion width (measured)
SEED_TFXY = 1003
HBM_FALLBACK = 6800.0


def aggregate_ranks(elapsed_s: float, units_per_rank: float, dist=None, device="cpu"):
    """Replicas: every rank processes `units_per_rank`; the job's time is the
    slowest rank's.  Returns (max elapsed over ranks, total units / that time)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_s = float(t.item())
        dist.barrier()
    return elapsed_s, units_per_rank * world / elapsed_s


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return HBM_FALLBACK, "fallback"


def workload():
    rng = np.random.default_rng(SEED_BASIS)
    x = int(rng.integers(0, 1 << N_QUBITS))
    return x, C.qft(N_QUBITS), C.brickwork(N_QUBITS, BRICK_DEPTH, seed=SEED_BRICK)


def algorithmic_bytes(g, n, elem):
    """Read+write bytes a gate sweep must move (what it changes, nothing else)."""
    N = 1 << n
    name = g.name.upper()
    nc = len(g.controls)
    frac = 1.0 / (1 << nc)
    if name == "SWAP":
        return 2 * N * elem * 0.5 * frac
    if name in ("X",):
        return 2 * N * elem * frac
    if name in ("Z", "S", "SDG", "T", "TDG", "P"):
        return 2 * N * elem * 0.5 * frac
    return 2 * N * elem * frac


def sector_bytes(g, n, elem):
    """Read + write bytes of the 32-byte DRAM sectors that hold the amplitudes a
    gate changes.  A sector holds 32 / elem amplitudes that differ in the lowest
    one (complex128) or two (complex64) index bits, so a condition on those bits
    (a control, the pattern of a phase gate) does not reduce the sectors moved."""
    inb = 1 if elem == 16 else 2
    N = 1 << n
    pos = lambda qb: n - 1 - qb
    name = g.name.upper()
    cond = [pos(c) for c in g.controls]
    if name in ("Z", "S", "SDG", "T", "TDG", "P"):
        cond += [pos(t) for t in g.qubits]
    frac = 1.0
    if name == "SWAP":          # changed where the two bits differ
        a, b = pos(g.qubits[0]), pos(g.qubits[1])
        frac = 0.5 if (a >= inb and b >= inb) else 1.0
    return 2 * N * elem / (1 << sum(1 for p in cond if p >= inb)) * frac


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_sources_sha():
    """Fingerprint of the dense-sweep kernel: the arithmetic header and the
    k_dense section of qc_gates.cu (other kernels in the file do not count)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2303_00123_gb300", "csrc")
    h.update(open(os.path.join(csrc, "qc_common.cuh"), "rb").read())
    g = open(os.path.join(csrc, "qc_gates.cu")).read()
    a = g.index("// ---------------------------------------------------------------- dense")
    b = g.index("// ---------------------------------------------------------------- permutation")
    h.update(g[a:b].encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the dense 1-qubit kernel from the committed
    ncu summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "dense1q_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("src_sha") != kernel_sources_sha():
        return None
    return d.get("dram_bytes_per_launch")


# ---------------------------------------------------------------- CPU oracle
def gate_class(g):
    """Cost class of a gate for extrapolating oracle timings."""
    name = g.name.upper()
    if name == "SWAP":
        return "swap"
    if g.controls:
        return "controlled"
    return "one_qubit"


def oracle_sample_gates():
    """40 gates of the step that cover every gate class: the first 14 and the
    last 3 (SWAP) of the QFT, the first 20 Haar U(2) and 3 CNOTs of the brickwork."""
    x, qft, brick = workload()
    cnots = [g for g in brick if g.controls][:3]
    return x, qft[:14] + qft[-3:] + brick[:20] + cnots, qft + brick


def cpu_oracle_sample():
    """The FP64 oracle (C, OpenMP over the host cores) on 40 gates of the step
    at n=30, extrapolated to the whole step per gate class; plus the oracle on
    one thread for two gates (a U(2) and a controlled phase), scaled by class."""
    from oracle import oracle as O
    x, sample, full = oracle_sample_gates()
    psi = O.basis_state(N_QUBITS, x)
    per = {}
    t_all = time.perf_counter()
    for g in sample:
        t0 = time.perf_counter()
        O.apply_gate(psi, N_QUBITS, g)
        per.setdefault(gate_class(g), []).append(time.perf_counter() - t0)
    dt = time.perf_counter() - t_all
    del psi
    cls_s = {c: float(np.mean(v)) for c, v in per.items()}
    step_s = sum(cls_s[gate_class(g)] for g in full)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": round(len(full) / step_s, 4), "unit": "gates/s", "cores": cores, "kind": "oracle",
           "sample": "40 of the step's gates at n=%d complex128 (QFT: first 14 and the 3 last SWAPs; brickwork: "
                     "first 20 U(2) and 3 CNOTs), %.1f s, extrapolated to the %d-gate step per gate class"
                     % (N_QUBITS, dt, len(full)),
           "sample_gates_per_s": round(len(sample) / dt, 4),
           "s_per_gate_by_class": {c: round(v, 4) for c, v in cls_s.items()}}
    # single thread: the oracle library reads OMP_NUM_THREADS at load; run it in a child process
    code = ("import sys, time, json; sys.path.insert(0, %r); import bench; from oracle import oracle as O;"
            "x, sample, full = bench.oracle_sample_gates(); g1 = [g for g in sample if bench.gate_class(g) == "
            "'one_qubit'][0]; g2 = [g for g in sample if bench.gate_class(g) == 'controlled'][0];"
            "psi = O.basis_state(bench.N_QUBITS, x); r = {};"
            "t0 = time.perf_counter(); O.apply_gate(psi, bench.N_QUBITS, g1); r['one_qubit'] = time.perf_counter() - t0;"
            "t0 = time.perf_counter(); O.apply_gate(psi, bench.N_QUBITS, g2); r['controlled'] = time.perf_counter() - t0;"
            "print(json.dumps(r))" % ROOT)
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        one = json.loads(r.stdout.strip().splitlines()[-1])
        # classes not timed on one thread take the multithreaded ratio of the U(2) gate
        ratio = one["one_qubit"] / cls_s["one_qubit"]
        st_s = sum(one.get(gate_class(g), cls_s[gate_class(g)] * ratio) for g in full)
        out["single_thread"] = {"value": round(len(full) / st_s, 5), "unit": "gates/s", "cores": 1,
                                "sample": "one U(2) and one controlled phase at n=30 on one thread, "
                                          "extrapolated to the step per gate class",
                                "s_per_gate_by_class": {c: round(v, 3) for c, v in one.items()}}
    except Exception as e:  # noqa: BLE001 -- the multithreaded figure stands alone
        out["single_thread"] = {"unavailable": str(e)[:200]}
    return out


def workload_config(args, world, gates_per_step):
    """The `config` both arms report: the same workload, whichever arm runs it."""
    return {"workload": "n=30 complex128 QFT (seeded basis state) + brickwork depth 40 (Haar U(2) "
                        "layers + CNOT pairs), gate by gate", "n": N_QUBITS, "gates_per_step": gates_per_step,
            "fuse_k": args.fuse, "arith": args.arith, "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (17.2 GB state vs 129 MB)"}


# ---------------------------------------------------------------- GPU arm
E2E_MAX_STEPS = 3        # the end-to-end loop repeats at most this many steps


def dense_roofline(ms_list, bytes_total, peak, peak_kind, label, traffic=None):
    """Roofline of the dense 1-qubit sweep from per-launch CUDA-event times."""
    if not ms_list:
        return None
    per_launch_bytes = bytes_total / len(ms_list)
    avg_ms = float(np.mean(ms_list))
    achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": label,
            "peak_kind": peak_kind + " (copy bandwidth, MEASURED_PEAKS.json)",
            "algorithmic_bytes_per_launch": per_launch_bytes, "avg_launch_ms": round(avg_ms, 4),
            "launches": len(ms_list)}


def run_gpu(args):
    import torch
    from paper_2303_00123_gb300 import qcgb300 as q

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = N_QUBITS
    x, qft, brick = workload()
    gates_per_step = len(qft) + len(brick)
    t = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    st = q.State.from_tensor(t)
    arith = q.ARITH_F32X2 if args.arith == "f32x2" else q.ARITH_NATIVE
    st.set_arith(arith)
    stream = torch.cuda.Stream()
    st.set_stream(stream)
    elem = 16

    dense_ms, dense_bytes = [], 0.0
    per_q = {}
    launches = 0

    def step(record, sink=None):
        nonlocal launches, dense_bytes
        for circ in (qft, brick):
            st.set_basis(x)
            nl, ms = st.apply_circuit(circ, fuse_k=args.fuse, time_gates=record)
            launches += nl
            if record and args.fuse == 0:
                for g, m in zip(circ, ms):
                    if g.name.upper() == "U" and not g.controls:
                        (sink if sink is not None else dense_ms).append(m)
                        if sink is None:
                            dense_bytes += algorithmic_bytes(g, n, elem)
                            per_q.setdefault(g.qubits[0], []).append(m)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    launches = 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step(True)
        ev1.record(stream)
        torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    elapsed, value = aggregate_ranks(elapsed, gates_per_step * args.steps, dist, "cuda")

    peak, peak_kind = measured_peaks()
    roof = dense_roofline(dense_ms, dense_bytes, peak, peak_kind,
                          "k_dense (1-qubit Haar U(2), complex128, %s)" % args.arith, profiled_traffic())
    per_target = None
    if per_q:
        ub = 2 * (1 << n) * elem
        per_target = {"what": "dense 1-qubit Haar U(2) sweeps of the brickwork, by target qubit q (stride 2^(29-q) "
                              "amplitudes): average GB/s of algorithmic bytes",
                      "q": sorted(per_q), "GBps": [round(ub / (float(np.mean(per_q[k])) * 1e-3) / 1e9, 1)
                                                   for k in sorted(per_q)]}

    # the same step in native FP64 arithmetic (one timed step, outside the timed region)
    native = None
    if not args.no_native and args.arith == "f32x2" and args.fuse == 0:
        st.set_arith(q.ARITH_NATIVE)
        for circ in (qft, brick):          # warm the native kernels on a few gates of each circuit
            st.set_basis(x)
            st.apply_circuit(circ[:40])
        nat_ms = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        step(True, sink=nat_ms)
        e1.record(stream)
        torch.cuda.synchronize()
        nat_s = e0.elapsed_time(e1) / 1e3
        st.set_arith(arith)
        native = {"value": round(gates_per_step / nat_s, 3), "unit": "gates/s", "dtype": "c128-f64",
                  "ms_per_step": round(nat_s * 1e3, 1), "steps": 1,
                  "roofline": dense_roofline(nat_ms, 2 * (1 << n) * elem * len(nat_ms), peak, peak_kind,
                                             "k_dense (1-qubit Haar U(2), complex128, native FP64)"),
                  "note": "the same step with QC_ARITH_NATIVE: plain FP64 arithmetic (GB300 FP64 FMA ~1/64 of FP32)"}

    # e2e through the C ABI with pinned host buffers: the input state (prepared once) is
    # copied host->device for every circuit, the final state device->host into a second buffer
    e2e = None
    if not args.no_e2e:
        # page-locked, huge-page host buffers (qcgb300.HostBuffer): the input state and the result
        host_in = q.HostBuffer(1 << n, np.complex128)
        host_in.array[x] = 1.0
        host_out = q.HostBuffer(1 << n, np.complex128)
        in_np, out_np = host_in.array, host_out.array
        huge = [host_in.huge_page_bytes(), host_out.huge_page_bytes()]
        e2e_steps = max(1, min(args.steps, E2E_MAX_STEPS))
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(2 * e2e_steps)]
        enqueue_s = 0.0
        # the first copy from the freshly registered input buffer, on its own, before the timed loop
        # (diagnostic: it includes the first translations of the buffer's pages)
        torch.cuda.synchronize()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        q.lib.qc_state_copy_from_host(st.handle, q.ctypes.c_void_p(in_np.ctypes.data))
        eb.record(stream)
        torch.cuda.synchronize()
        h2d_first = ea.elapsed_time(eb)
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            for c, circ in enumerate((qft, brick)):
                ev = evs[2 * i + c]
                ev[0].record(stream)
                q.lib.qc_state_copy_from_host(st.handle, q.ctypes.c_void_p(in_np.ctypes.data))
                ev[1].record(stream)
                ta = time.perf_counter()
                st.apply_circuit(circ, fuse_k=args.fuse)
                enqueue_s += time.perf_counter() - ta
                ev[2].record(stream)
                st.to_numpy(out=out_np)     # device->host copy of the final state (synchronises)
                ev[3].record(stream)
        e2e_s = time.perf_counter() - t0
        torch.cuda.synchronize()
        h2d_each = [round(e[0].elapsed_time(e[1]), 1) for e in evs]
        h2d = sum(e[0].elapsed_time(e[1]) for e in evs) / e2e_steps
        circ_ms = sum(e[1].elapsed_time(e[2]) for e in evs) / e2e_steps
        d2h = sum(e[2].elapsed_time(e[3]) for e in evs) / e2e_steps
        wall = e2e_s / e2e_steps * 1e3
        del in_np, out_np
        host_in.free()
        host_out.free()
        bi = 2 * (1 << n) * elem
        e2e = {"value": gates_per_step * e2e_steps * world / e2e_s, "unit": "gates/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bi, "steps": e2e_steps,
               "breakdown_ms_per_step": {
                   "wall": round(wall, 1), "h2d": round(h2d, 1), "circuits": round(circ_ms, 1), "d2h": round(d2h, 1),
                   "host_enqueue": round(enqueue_s / e2e_steps * 1e3, 1),
                   "other": round(wall - h2d - circ_ms - d2h, 1),
                   "h2d_each_ms": h2d_each, "h2d_first_ms": round(h2d_first, 1),
                   "host_buffers": "page-locked, transparent huge pages (qcgb300.HostBuffer)",
                   "huge_page_bytes_in_out": huge,
                   "note": "h2d, circuits, d2h: CUDA events on the state's stream around each phase (two circuits "
                           "per step); host_enqueue: wall time of the apply calls (marshalling, planning, launches, "
                           "overlapping the device work); other = wall - h2d - circuits - d2h"}}

    extras = {} if args.no_extras else extra_measurements(q, st, stream, brick, x, args)
    line = {
        "metric": "gates/s at n=30 complex128 (QFT 480 + brickwork depth-40 1780 gates, unfused)",
        "value": round(value, 3), "unit": "gates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed / args.steps * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128-" + args.arith, "data": "synthetic",
        "arith_note": ("complex128 state (IEEE binary64 in HBM); each gate computed in float-float on the FP32 pipes "
                       "(47-bit significands, inputs below 2^-100 flushed); native_fp64 below is the same step in "
                       "plain FP64" if args.arith == "f32x2" else "plain FP64 arithmetic"),
        "config": workload_config(args, world, gates_per_step),
        "gpu_launches": launches,
        "roofline": roof,
        "e2e": e2e,
        "clocks": clk.summary(),
    }
    if native:
        line["native_fp64"] = native
    if per_target:
        line["per_target"] = per_target
    line.update(extras)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_sample()
    st.free()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def case_gates(kind, n, rng):
    """One gate per target position for the --case micro-benchmarks."""
    gates = []
    for t in range(n):
        if kind == "dense1q":
            gates.append(C.Gate("U", (t,), matrix=C.haar_unitary(rng, 2)))
        elif kind == "cnot":
            gates.append(C.Gate("X", (t,), controls=((t + 1) % n,)))
        elif kind == "cphase":
            gates.append(C.Gate("P", (t,), controls=((t + 7) % n,), theta=0.3))
        elif kind == "dense2q":
            gates.append(C.Gate("U4", (t, (t + 1) % n), matrix=C.haar_unitary(rng, 4)))
        elif kind == "swap":
            gates.append(C.Gate("SWAP", (t, (t + n // 2) % n)))
        elif kind == "h":
            gates.append(C.Gate("H", (t,)))
        elif kind.startswith("kq"):
            k = int(kind[2:])
            qs = [(t + 3 * i) % n for i in range(k)]
            if len(set(qs)) < k:
                continue
            gates.append(C.Gate("UK", tuple(qs), matrix=C.haar_unitary(rng, 1 << k)))
        else:
            raise SystemExit("unknown case " + kind)
    return gates


def run_adjoint_case(args):
    """Adjoint gradients of the hardware-efficient ansatz (n qubits, 10
    layers of RY, RZ and a CNOT ladder, 2*n*10 parameters) for the TFIM chain,
    a batch of parameter sets per call; reports gradient sets per second."""
    import torch
    from paper_2303_00123_gb300 import qcgb300 as q
    n, layers, B = args.n, 10, args.batch
    th = C.hea_thetas(n, layers, seed=2025, batch=B)
    gates = C.hea(n, layers, th[0])
    H = C.tfim(n, 1.0)
    dt = q.C64 if args.dtype == "c64" else q.C128
    ar = q.ARITH_F32X2 if args.arith == "f32x2" else q.ARITH_NATIVE
    for _ in range(args.warmup):
        q.adjoint_grad(n, gates, H, th, dtype=dt, arith=ar)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e, g = q.adjoint_grad(n, gates, H, th, dtype=dt, arith=ar)
    dt_s = (time.perf_counter() - t0) / args.steps
    state_bytes = (1 << n) * (8 if dt == q.C64 else 16)
    nparam = g.shape[1]
    print(json.dumps({"case": "adjoint", "n": n, "layers": layers, "batch": B, "params": nparam,
                      "dtype": args.dtype, "arith": args.arith, "s_per_call": round(dt_s, 4),
                      "gradient_sets_per_s": round(B / dt_s, 2),
                      "param_grads_per_s": round(B * nparam / dt_s, 1),
                      "workspace_bytes": 2 * B * state_bytes}))


def run_batch_case(args):
    """1024 independent random circuits (n ~ U[10,24], depth ~ U[50,300],
    complex64) in one persistent launch (autotuned fusion, graph replay)
    against one circuit after another with one launch per gate."""
    import torch
    from paper_2303_00123_gb300 import qcgb300 as q
    specs = C.batch_specs(args.batch, seed=4)
    circs = [C.random_mix(n, d, seed=s) for n, d, s in specs]
    ngates = sum(len(g) for g in circs)
    dt = q.C64 if args.dtype == "c64" else q.C128
    sts = [q.State(n, dt) for n, _, _ in specs]
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    b = q.Batch(sts, circs, fuse_k=args.fuse if args.fuse != 0 else -1, use_graph=True, stream=stream)
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        b.launch(timing=True)
    tots, comps = [], []
    for _ in range(args.steps):
        comp, tot = b.launch(timing=True)
        tots.append(tot)
        comps.append(comp)
    tot = float(np.median(tots))
    comp = comps[int(np.argmin(np.abs(np.array(tots) - tot)))]
    info = b.info()
    b.free()
    # baseline: one circuit after another, one launch per gate
    for st in sts:
        st.set_stream(stream)
    base_comp = np.zeros(len(circs))
    ev0 = torch.cuda.Event(enable_timing=True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in circs]
    for rep in range(2):                 # first pass warms up
        ev0.record(stream)
        for i, (st, g) in enumerate(zip(sts, circs)):
            st.set_basis(0)
            st.apply_circuit(g)
            evs[i].record(stream)
        stream.synchronize()
    for i in range(len(circs)):
        base_comp[i] = ev0.elapsed_time(evs[i])
    base_tot = float(base_comp.max())
    for st in sts:
        st.free()
    print(json.dumps({"case": "batch", "circuits": len(circs), "gates": ngates, "dtype": args.dtype,
                      "fuse_k": info["fuse_k"], "ops": info["ops"], "smem_circuits": info["smem_circuits"],
                      "persistent": {"ms": round(tot, 3), "gates_per_s": round(ngates / tot * 1e3, 1),
                                     "p50_ms": round(float(np.percentile(comp, 50)), 3),
                                     "p99_ms": round(float(np.percentile(comp, 99)), 3)},
                      "one_launch_per_gate": {"ms": round(base_tot, 3), "gates_per_s": round(ngates / base_tot * 1e3, 1),
                                              "p50_ms": round(float(np.percentile(base_comp, 50)), 3),
                                              "p99_ms": round(float(np.percentile(base_comp, 99)), 3)},
                      "speedup": round(base_tot / tot, 2), "autotune_s": round(tune_s, 2)}))


def circuit_for(name, n):
    """Benchmark circuit families: QFT, brickwork depth 40, TFXY Trotter (10 steps)."""
    if name == "qft":
        return C.qft(n)
    if name == "tfxy":
        return C.tfxy_trotter(n, TFXY_STEPS, seed=SEED_TFXY)
    return C.brickwork(n, BRICK_DEPTH, seed=SEED_BRICK)


def run_fused_case(args):
    """Brickwork depth 40 at n qubits with greedy fusion k = 0 (gate by gate),
    2, 3, 4, 5: time, launches, gates/s, and effective HBM GB/s (sum of the
    launches' algorithmic bytes 2*N*E / time); amplitude error against the
    FP64 oracle on the same circuit family at n_err qubits."""
    import torch
    from paper_2303_00123_gb300 import qcgb300 as q
    n = args.n
    dt = q.C64 if args.dtype == "c64" else q.C128
    elem = 8 if dt == q.C64 else 16
    gates = circuit_for(args.circuit, n)
    t = torch.empty(1 << n, dtype=torch.complex64 if dt == q.C64 else torch.complex128, device="cuda")
    st = q.State.from_tensor(t)
    st.set_arith(q.ARITH_F32X2 if args.arith == "f32x2" else q.ARITH_NATIVE)
    st.set_fused_tc(0 if args.no_tc else args.tc_mode)
    stream = torch.cuda.Stream()
    st.set_stream(stream)
    res = {}
    ks = (args.fuse,) if args.fuse else (0, 2, 3, 4, 5)   # --fuse K: that width only
    for k in ks:
        for _ in range(args.warmup):
            st.set_basis(0)
            st.apply_circuit(gates, fuse_k=k)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            st.set_basis(0)
            nl, _ = st.apply_circuit(gates, fuse_k=k)
        ev1.record(stream)
        stream.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        res[str(k)] = {"ms": round(ms, 2), "launches": nl, "gates_per_s": round(len(gates) / ms * 1e3, 1),
                       "eff_GBps": round(nl * 2 * (1 << n) * elem / (ms * 1e-3) / 1e9, 1)}
    st.free()
    del t
    torch.cuda.empty_cache()
    # accuracy against the oracle at n_err
    err = {}
    if args.n_err > 0:
        from oracle import oracle as O
        ne = args.n_err
        g2 = circuit_for(args.circuit, ne)
        ref = O.run_circuit(ne, g2)
        for k in ks:
            s2 = q.State(ne, dt)
            s2.set_arith(q.ARITH_F32X2 if args.arith == "f32x2" else q.ARITH_NATIVE)
            s2.set_fused_tc(0 if args.no_tc else args.tc_mode)
            s2.apply_circuit(g2, fuse_k=k)
            got = s2.to_numpy().astype(np.complex128)
            s2.free()
            err[str(k)] = {"max_abs": float(np.max(np.abs(got - ref))),
                           "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}
    print(json.dumps({"case": "fused", "circuit": args.circuit, "n": n, "dtype": args.dtype, "arith": args.arith,
                      "gates": len(gates),
                      "tensor_cores": (not args.no_tc) and (args.dtype == "c64" or args.arith == "f32x2"),
                      "by_fuse_k": res, "n_err": args.n_err, "error_vs_oracle": err,
                      "speedup_best_vs_unfused": (round(res["0"]["ms"] / min(v["ms"] for v in res.values()), 2)
                                                  if "0" in res else None)}))


def run_expect_case(args):
    """qc_expect of the TFIM chain (n-1 ZZ terms, n X terms) on a seeded
    n-qubit state: time, and GB/s against the passes the plan makes (each pass
    reads the whole state once).  For comparison the one-sweep-per-flip-mask
    form (qc_expect_noalloc: 1 + n sweeps) is timed on the same state."""
    import torch
    from paper_2303_00123_gb300 import qcgb300 as q
    n = args.n
    dt = q.C64 if args.dtype == "c64" else q.C128
    elem = 8 if dt == q.C64 else 16
    st = q.State(n, dt)
    st.apply_circuit([C.Gate("H", (i,)) for i in range(n)] + C.random_mix(n, 20, seed=3))
    H = C.tfim(n, 1.0)
    passes = q.expect_passes(n, dt, H)

    def timed(f):
        for _ in range(args.warmup):
            f(H)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            v = f(H)
        return (time.perf_counter() - t0) / args.steps, v

    t_tile, e = timed(st.expect)
    t_sweep, e2 = timed(st.expect_noalloc)
    state_gb = (1 << n) * elem / 1e9
    gbps = passes * state_gb / t_tile
    peak, _ = measured_peaks()
    print(json.dumps({"case": "expect", "n": n, "dtype": args.dtype, "terms": len(H), "passes": passes,
                      "ms": round(t_tile * 1e3, 3), "GBps": round(gbps, 1),
                      "frac_of_measured_hbm": round(gbps / peak, 4),
                      "one_read_floor_ms": round(state_gb / peak * 1e3, 3),
                      "per_flip_sweeps": {"sweeps": 1 + n, "ms": round(t_sweep * 1e3, 3)},
                      "speedup": round(t_sweep / t_tile, 2), "energy": e, "energy_sweeps": e2}))
    st.free()


def run_shard_case(args):
    """One n-qubit state as 2^g shards on this GPU (every shard its own state):
    the QFT and a depth-10 brickwork through the exchange plan, against the
    unsharded state; exchanges are in-place kernels trading half of each of two
    shards (every shard's half read and written: N * E bytes per exchange step)."""
    import torch
    from paper_2303_00123_gb300 import qcgb300 as q, shard
    n, g = args.n, args.g
    dt = q.C64 if args.dtype == "c64" else q.C128
    elem = 8 if dt == q.C64 else 16
    stream = torch.cuda.current_stream()
    out = {"case": "shard", "n": n, "g": g, "dtype": args.dtype}
    for name, circ in (("qft", C.qft(n)), ("brickwork10", C.brickwork(n, 10, seed=SEED_BRICK))):
        steps = shard.plan(n, g, circ)
        nex = sum(1 for st in steps if st[0] == "exchange")
        states = [q.State(n - g, dt) for _ in range(1 << g)]
        for st in states:
            st.set_stream(stream)

        def sharded():
            # timing only: shard 0 restarts from its basis state, the other shards keep
            # whatever the previous run left (the sweeps' cost does not depend on the values)
            states[0].set_basis(0)
            shard.run_single_device(states, n, g, steps)
        sharded()
        ms = _event_ms(stream, sharded)
        # the exchanges alone: one per step, on the basis state
        ex = [st_ for st_ in steps if st_[0] == "exchange"]

        def exchanges():
            for _, bit, local in ex:
                for r in range(1 << g):
                    if (r >> bit) & 1 == 0:
                        q.shard_exchange(states[r], states[r ^ (1 << bit)], local, 0)
        ex_ms = _event_ms(stream, exchanges) if ex else 0.0
        for st in states:
            st.free()
        whole = q.State(n, dt)
        whole.set_stream(stream)

        def unsharded():
            whole.set_basis(0)
            whole.apply_circuit(circ)
        unsharded()
        ms0 = _event_ms(stream, unsharded)
        whole.free()
        torch.cuda.empty_cache()
        peak, _ = measured_peaks()
        exb = (1 << n) * elem * len(ex)     # each exchange reads and writes half of every shard
        out[name] = {"gates": len(circ), "exchanges": nex, "sharded_ms": round(ms, 1), "unsharded_ms": round(ms0, 1),
                     "exchange_ms": round(ex_ms, 1),
                     "exchange_GBps": round(exb / (ex_ms * 1e-3) / 1e9, 1) if ex_ms else None,
                     "exchange_frac_of_measured_hbm": round(exb / (ex_ms * 1e-3) / 1e9 / peak, 4) if ex_ms else None}
    print(json.dumps(out))


def run_case(args):
    """Per-target-qubit timing of one gate kind on an n-qubit state."""
    import torch
    from paper_2303_00123_gb300 import qcgb300 as q
    if args.case == "expect":
        return run_expect_case(args)
    if args.case == "adjoint":
        return run_adjoint_case(args)
    if args.case == "batch":
        return run_batch_case(args)
    if args.case == "fused":
        return run_fused_case(args)
    if args.case == "shard":
        return run_shard_case(args)
    n = args.n
    dt = q.C64 if args.dtype == "c64" else q.C128
    elem = 8 if dt == q.C64 else 16
    t = torch.zeros(1 << n, dtype=torch.complex64 if dt == q.C64 else torch.complex128, device="cuda")
    st = q.State.from_tensor(t)
    st.set_arith(q.ARITH_F32X2 if args.arith == "f32x2" else q.ARITH_NATIVE)
    st.set_fused_tc(0 if args.no_tc else args.tc_mode)
    st.set_packed(args.packed)
    stream = torch.cuda.Stream()
    st.set_stream(stream)
    st.set_basis(0)
    gates = case_gates(args.case, n, np.random.default_rng(7))
    for _ in range(args.warmup):
        st.apply_circuit(gates)
    per = np.zeros(len(gates))
    for _ in range(args.steps):
        _, ms = st.apply_circuit(gates, time_gates=True)
        per += ms
    per /= max(1, args.steps)
    out = []
    for g, m in zip(gates, per):
        b = algorithmic_bytes(g, n, elem)
        out.append({"q": g.qubits[0], "qubits": list(g.qubits), "stride": 1 << (n - 1 - g.qubits[0]), "ms": round(float(m), 4),
                    "GBps": round(b / (m * 1e-3) / 1e9, 1),
                    "GBps_sector": round(sector_bytes(g, n, elem) / (m * 1e-3) / 1e9, 1)})
    peak, _ = measured_peaks()
    tot_b = sum(algorithmic_bytes(g, n, elem) for g in gates)
    tot_s = sum(sector_bytes(g, n, elem) for g in gates)
    print(json.dumps({"case": args.case, "n": n, "dtype": args.dtype, "arith": args.arith, "tc": not args.no_tc,
                      "packed": args.packed,
                      "avg_GBps": round(tot_b / (per.sum() * 1e-3) / 1e9, 1),
                      "frac_of_measured_hbm": round(tot_b / (per.sum() * 1e-3) / 1e9 / peak, 4),
                      "avg_GBps_sector": round(tot_s / (per.sum() * 1e-3) / 1e9, 1),
                      "frac_sector": round(tot_s / (per.sum() * 1e-3) / 1e9 / peak, 4),
                      "per_target": out}))
    st.free()


def _event_ms(stream, fn, reps=1):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    stream.synchronize()
    return e0.elapsed_time(e1) / reps


def fusion_sweep(q, stream, brick, peak):
    """Brickwork depth 40 fused into k-qubit blocks: n=30 complex128 and
    complex64 at k = 0 (gate by gate), 2, 3, 4, 5; n=32 at k = 5; amplitude
    error against the FP64 oracle at n=20 for every k.  Tensor-core blocks
    (k >= 3): algorithmic flops 8 * 2^k per amplitude and block over the
    tensor peak of the operand type (tf32 = bf16 / 2, fp16 = bf16, nominal
    ratios), beside the HBM fraction."""
    import torch
    from oracle import oracle as O
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    out = {}
    # warm every kernel shape on a small state first (function attributes, first launches)
    for dt in (q.C128, q.C64):
        sw = q.State(20, dt)
        sw.set_stream(stream)
        for k in (0, 2, 3, 4, 5):
            sw.set_basis(0)
            sw.apply_circuit(C.brickwork(20, 4, seed=1), fuse_k=k)
        sw.free()
    for n, ks in ((N_QUBITS, (0, 2, 3, 4, 5)), (32, (5,))):
        circ = brick if n == N_QUBITS else C.brickwork(n, BRICK_DEPTH, seed=SEED_BRICK)
        for dname, dt, elem, tdt in (("c128", q.C128, 16, torch.complex128), ("c64", q.C64, 8, torch.complex64)):
            t = torch.empty(1 << n, dtype=tdt, device="cuda")
            s2 = q.State.from_tensor(t)
            s2.set_stream(stream)
            res = {}
            for k in ks:
                def run():
                    s2.set_basis(0)
                    s2.apply_circuit(circ, fuse_k=k)
                ms = _event_ms(stream, run)
                plan = q.fuse_plan(n, circ, k) if k else None
                nl = len(plan) if k else len(circ)
                nblk = sum(1 for b in plan if not isinstance(b[0], str) and len(b[0]) >= 3) if k >= 3 else 0
                if k:   # a block sweep moves 2 N E bytes (halved per control)
                    byts = sum(2 * (1 << n) * elem / (1 << len(b[1])) if not isinstance(b[0], str)
                               else 2 * (1 << n) * elem for b in plan)
                else:
                    byts = sum(algorithmic_bytes(gt, n, elem) for gt in circ)
                hbm = byts / (ms * 1e-3) / 1e9
                r = {"ms": round(ms, 1), "launches": nl, "gates_per_s": round(len(circ) / ms * 1e3, 1),
                     "eff_GBps": round(hbm, 1), "hbm_frac": round(hbm / peak, 4)}
                if nblk:
                    tpeak = bf16 / 2 if dt == q.C64 else bf16
                    tf = nblk * 8 * (1 << k) * (1 << n) / (ms * 1e-3) / 1e12
                    r["tensor"] = {"blocks": nblk, "TFLOPs": round(tf, 1), "peak": round(tpeak, 1),
                                   "frac": round(tf / tpeak, 4),
                                   "op": "tf32 split (3 products)" if dt == q.C64 else "fp16 digit slices (27 products)"}
                res[str(k)] = r
            if "0" in res:
                res["speedup_k5"] = round(res["0"]["ms"] / res["5"]["ms"], 2)
            out["n%d_%s" % (n, dname)] = res
            s2.free()
            del t
            torch.cuda.empty_cache()
    # accuracy at n=20 against the FP64 oracle (same circuit family)
    ne = 20
    g2 = C.brickwork(ne, BRICK_DEPTH, seed=SEED_BRICK)
    ref = O.run_circuit(ne, g2)
    err = {}
    for dname, dt in (("c128", q.C128), ("c64", q.C64)):
        for k in (0, 2, 3, 4, 5):
            s3 = q.State(ne, dt)
            s3.apply_circuit(g2, fuse_k=k)
            got = s3.to_numpy().astype(np.complex128)
            s3.free()
            err["%s_k%d" % (dname, k)] = {"max_abs": float(np.max(np.abs(got - ref))),
                                           "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}
    out["error_vs_oracle_n20"] = err
    return out


def extra_measurements(q, st, stream, brick, x, args):
    """Fused, batched and adjoint forms against the plain per-gate form, on
    this GPU, outside the main timed region (each reported with its config)."""
    import torch
    out = {}
    peak, _ = measured_peaks()
    fused = {"brickwork": fusion_sweep(q, stream, brick, peak)}
    qft = C.qft(N_QUBITS)
    def qft_run(k):
        st.set_basis(x)
        st.apply_circuit(qft, fuse_k=k)
    qft_run(2)
    q0 = _event_ms(stream, lambda: qft_run(0))
    q2 = _event_ms(stream, lambda: qft_run(2))
    fused["qft_c128_k2"] = {"ms": round(q2, 1), "unfused_ms": round(q0, 1), "speedup": round(q0 / q2, 2),
                            "launches": len(q.fuse_plan(N_QUBITS, qft, 2))}
    # expectation of the TFIM chain on the same 30-qubit state: tiled passes vs
    # one sweep per distinct flip mask
    Ht = C.tfim(N_QUBITS, 1.0)
    st.expect(Ht)
    te0 = time.perf_counter()
    for _ in range(3):
        e_tile = st.expect(Ht)
    te_tile = (time.perf_counter() - te0) / 3 * 1e3
    st.expect_noalloc(Ht)
    te0 = time.perf_counter()
    for _ in range(2):
        e_sweep = st.expect_noalloc(Ht)
    te_sweep = (time.perf_counter() - te0) / 2 * 1e3
    passes = q.expect_passes(N_QUBITS, q.C128, Ht)
    peak, _ = measured_peaks()
    gb = passes * (1 << N_QUBITS) * 16 / 1e9
    out["expect"] = {"workload": "TFIM chain (29 ZZ + 30 X terms), n=30 complex128", "passes": passes,
                     "ms": round(te_tile, 2), "GBps": round(gb / te_tile * 1e3, 1),
                     "frac_of_measured_hbm": round(gb / te_tile * 1e3 / peak, 4),
                     "per_flip_mask_sweeps_ms": round(te_sweep, 1), "speedup": round(te_sweep / te_tile, 2),
                     "abs_diff": abs(e_tile - e_sweep)}
    t64 = torch.empty(1 << N_QUBITS, dtype=torch.complex64, device="cuda")
    s64 = q.State.from_tensor(t64)
    s64.set_stream(stream)
    # TFXY Trotter circuit (Sec. 4, 10 steps): complex128 k=2, complex64 k=5 on the tensor cores
    tfxy = C.tfxy_trotter(N_QUBITS, TFXY_STEPS, seed=SEED_TFXY)
    def tfxy_run(state, k):
        state.set_basis(0)
        state.apply_circuit(tfxy, fuse_k=k)
    tfxy_run(s64, 5)
    v0 = _event_ms(stream, lambda: tfxy_run(s64, 0))
    v5 = _event_ms(stream, lambda: tfxy_run(s64, 5))
    fused["tfxy_c64_k5_tensor_cores"] = {"ms": round(v5, 1), "unfused_ms": round(v0, 1), "speedup": round(v0 / v5, 2),
                                         "launches": len(q.fuse_plan(N_QUBITS, tfxy, 5))}
    s64.free()
    del t64
    torch.cuda.empty_cache()
    tfxy_run(st, TFXY_C128_K)
    w0 = _event_ms(stream, lambda: tfxy_run(st, 0))
    wk = _event_ms(stream, lambda: tfxy_run(st, TFXY_C128_K))
    fused["tfxy_c128_k%d" % TFXY_C128_K] = {"ms": round(wk, 1), "unfused_ms": round(w0, 1), "speedup": round(w0 / wk, 2),
                                            "launches": len(q.fuse_plan(N_QUBITS, tfxy, TFXY_C128_K))}
    out["fused"] = {"workload": "brickwork depth 40 (greedy k-qubit blocks) at n=30 (k=0,2..5) and n=32 (k=5), "
                                "complex128 and complex64, error vs the FP64 oracle at n=20; n=30 QFT (each H merged "
                                "with its phase run, final SWAPs as one bit permutation); n=30 TFXY Trotter, 10 steps",
                    **fused}
    # batched: 1024 circuits, one persistent launch vs one launch per gate, and vs
    # per-circuit fused launches spread over 8 streams
    specs = C.batch_specs(1024, seed=4)
    circs = [C.random_mix(n, d, seed=sd) for n, d, sd in specs]
    ngates = sum(len(g) for g in circs)
    sts = [q.State(n, q.C64) for n, _, _ in specs]
    t0 = time.perf_counter()
    b = q.Batch(sts, circs, fuse_k=-1, use_graph=True, stream=stream)
    tune_s = time.perf_counter() - t0
    b.launch(timing=True)
    comp, tot = b.launch(timing=True)
    info = b.info()
    b.free()
    # algorithmic bytes: a shared-memory circuit writes its state once; a global
    # one reads and writes it per launch op (the persistent plan's fused ops)
    kk = info["fuse_k"]
    abytes = 0.0
    for (n_, _, _), g in zip(specs, circs):
        sb = (1 << n_) * 8
        abytes += sb if sb <= 64 * 1024 else 2 * sb * len(q.fuse_plan(n_, g, kk))
    for s2 in sts:
        s2.set_stream(stream)
    def one_by_one():
        for s2, g in zip(sts, circs):
            s2.set_basis(0)
            s2.apply_circuit(g)
    one_by_one()
    tb = _event_ms(stream, one_by_one)
    streams = [torch.cuda.Stream() for _ in range(8)]
    for i2, s2 in enumerate(sts):
        s2.set_stream(streams[i2 % 8])
    def fused_streams():
        for s2, g in zip(sts, circs):
            s2.set_basis(0)
            s2.apply_circuit(g, fuse_k=kk)
    fused_streams()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fused_streams()
    torch.cuda.synchronize()
    tf = (time.perf_counter() - t0) * 1e3
    for s2 in sts:
        s2.free()
    peak, _ = measured_peaks()
    out["batched"] = {"workload": "1024 random circuits, n~U[10,24], depth~U[50,300], complex64",
                      "gates": ngates, "persistent_ms": round(tot, 1), "gates_per_s": round(ngates / tot * 1e3, 1),
                      "p50_ms": round(float(np.percentile(comp, 50)), 1), "p99_ms": round(float(np.percentile(comp, 99)), 1),
                      "p50_over_makespan": round(float(np.percentile(comp, 50)) / tot, 3),
                      "roofline": {"bound": "hbm", "algorithmic_GB": round(abytes / 1e9, 2),
                                   "achieved": round(abytes / (tot * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                                   "frac": round(abytes / (tot * 1e-3) / 1e9 / peak, 4),
                                   "note": "shared-memory circuits: one state write; others: 2 N E per fused op; "
                                           "states below ~100 MB may stay in L2, so the fraction can exceed HBM's"},
                      "one_launch_per_gate_ms": round(tb, 1), "speedup": round(tb / tot, 2),
                      "fused_launches_8_streams_ms": round(tf, 1), "speedup_vs_fused_streams": round(tf / tot, 2),
                      "fuse_k": kk, "autotune_s": round(tune_s, 2)}
    # adjoint gradients vs parameter shift through the per-gate path (sampled, extrapolated)
    n, layers, B = 20, 10, 64
    th = C.hea_thetas(n, layers, seed=2025, batch=B)
    H = C.tfim(n, 1.0)
    gates = C.hea(n, layers, th[0])
    q.adjoint_grad(n, gates, H, th, dtype=q.C64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(2):
        q.adjoint_grad(n, gates, H, th, dtype=q.C64)
    ta = (time.perf_counter() - t0) / 2
    sp = q.State(n, q.C64)
    sp.set_stream(stream)
    def energy_eval():
        sp.set_basis(0)
        sp.apply_circuit(gates)
        return sp.expect(H)
    energy_eval()
    t0 = time.perf_counter()
    for _ in range(8):
        energy_eval()
    te = (time.perf_counter() - t0) / 8
    sp.free()
    nparam = 2 * n * layers
    ps_per_set = 2 * nparam * te
    out["adjoint"] = {"workload": "HEA n=20, 10 layers, 400 parameters, TFIM, batch 64, complex64 sweeps + FP64 reductions",
                      "s_per_batch": round(ta, 4), "gradient_sets_per_s": round(B / ta, 1),
                      "param_shift_s_per_set_extrapolated": round(ps_per_set, 3),
                      "speedup_vs_param_shift": round(ps_per_set / (ta / B), 1),
                      "note": "parameter shift timed as 8 energy evaluations (circuit + expectation) and scaled to 800"}
    return out


def run_reference(args):
    """The oracle as it stands, on the host cores: each step applies 6 gates of
    the 40-gate sample (in turn) to the n=30 state; `value` extrapolates the
    per-class times to the whole 2260-gate step."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    x, sample, full = oracle_sample_gates()
    psi = O.basis_state(N_QUBITS, x)
    for i in range(args.warmup):
        O.apply_gate(psi, N_QUBITS, sample[i % len(sample)])
    per = {}
    t_all = time.perf_counter()
    k = 0
    for _ in range(args.steps):
        for _ in range(6):
            g = sample[k % len(sample)]
            k += 1
            t0 = time.perf_counter()
            O.apply_gate(psi, N_QUBITS, g)
            per.setdefault(gate_class(g), []).append(time.perf_counter() - t0)
    dt = time.perf_counter() - t_all
    cls_s = {c: float(np.mean(v)) for c, v in per.items()}
    # classes the steps did not reach take the U(2) time (the costliest class)
    step_s = sum(cls_s.get(gate_class(g), cls_s.get("one_qubit", max(cls_s.values()))) for g in full)
    value = len(full) / step_s
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cpu = {"value": round(value, 4), "unit": "gates/s", "cores": cores, "kind": "oracle",
           "sample": "each step: 6 gates of a 40-gate sample of the n=30 complex128 step (QFT: first 14 and last 3 "
                     "SWAPs; brickwork: first 20 U(2), 3 CNOTs), taken in turn; extrapolated to the %d-gate step "
                     "per gate class" % len(full),
           "sample_gates_per_s": round(6 * args.steps / dt, 4)}
    cfg = workload_config(args, world, len(full))
    cfg["arith"] = "f64 (FP64 CPU oracle)"
    cfg["fuse_k"] = 0
    print(json.dumps({
        "impl": "reference", "metric": "gates/s at n=30 complex128 (QFT 480 + brickwork depth-40 1780 gates, unfused)",
        "value": round(value, 4), "unit": "gates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": cpu, "e2e": {"value": round(value, 4), "unit": "gates/s", "h2d_bytes_per_step": 0,
                                     "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--arith", default="f32x2", choices=["f32x2", "native"])
    ap.add_argument("--fuse", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-native", dest="no_native", action="store_true",
                    help="skip the native-FP64 step beside the float-float headline")
    ap.add_argument("--no-extras", dest="no_extras", action="store_true",
                    help="skip the fused / batched / adjoint side measurements")
    ap.add_argument("--case", default=None, help="micro-benchmark: dense1q, dense2q, cnot, cphase, swap, h")
    ap.add_argument("--n", type=int, default=28)
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--g", type=int, default=2, help="global qubits (--case shard)")
    ap.add_argument("--n-err", dest="n_err", type=int, default=0)
    ap.add_argument("--circuit", default="brickwork", choices=["brickwork", "qft", "tfxy"])
    ap.add_argument("--no-tc", dest="no_tc", action="store_true", help="complex64 blocks on CUDA cores")
    ap.add_argument("--tc-mode", dest="tc_mode", type=int, default=1, choices=[1, 2, 3, 4],
                    help="tensor-core block kernel (qc_set_fused_tc) of the micro-benchmarks")
    ap.add_argument("--packed", type=int, default=2, choices=[0, 1, 2],
                    help="complex128 float-float form: 0 scalar, 1 packed pairs, 2 packed + 2-qubit chains")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ and not args.case:
        # one replica rank per GPU, launched here when no launcher set the ranks up
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(args.gpus),
               "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
        raise SystemExit(subprocess.call(cmd))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world != args.gpus and not args.case:
        raise SystemExit("bench.py: --gpus %d but WORLD_SIZE=%d" % (args.gpus, world))
    if args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
