"""One state split over 2^g shards: running an exchange plan.

The plan comes from the library (``qc_shard_plan``): gate steps in shard qubit
numbering, each applied on the ranks whose bits match its global controls, and
exchange steps that trade half of every shard with a partner rank (a global
and a local qubit swap places).  This module walks a plan; the arithmetic and
the data movement on a GPU are the library's kernels:

* ``run_single_device``: all 2^g shards in one process (one GPU holds every
  shard as its own state), exchanges by ``qc_shard_exchange`` (one in-place
  kernel per pair of shards);
* ``run_rank``: one shard per process of a ``torch.distributed`` group (NCCL
  for GPUs), each exchange packing the outgoing half into a buffer
  (``qc_shard_pack``), trading buffers with the partner rank and unpacking
  (``qc_shard_unpack``).  The step walker takes a backend with ``apply``,
  ``pack``, ``empty_half`` and ``unpack``, so the same protocol runs with the
  GPU backend here or any other.
"""
from __future__ import annotations

from . import qcgb300 as q


def plan(n: int, g: int, gates):
    return q.shard_plan(n, g, gates)


def _gate_runs(steps):
    """Group consecutive gate steps: yields ("gates", [(gate, mask, val), ...])
    and ("exchange", rank_bit, local_qubit) items in plan order."""
    run = []
    for st in steps:
        if st[0] == "gate":
            run.append(st[1:])
            continue
        if run:
            yield ("gates", run)
            run = []
        yield st
    if run:
        yield ("gates", run)


def run_single_device(states, n: int, g: int, steps, fuse_k: int = 0):
    """Apply a plan to 2^g shard states held by this process (states[r] = rank
    r's shard, each of n - g qubits, on one device)."""
    if len(states) != 1 << g:
        raise q.QCError(q.QC_ERR_ARG, "need 2^g shard states")
    for item in _gate_runs(steps):
        if item[0] == "gates":
            for r, st in enumerate(states):
                mine = [gt for gt, mask, val in item[1] if (r & mask) == val]
                if mine:
                    st.apply_circuit(mine, fuse_k=fuse_k)
        else:
            _, bit, local = item
            for r in range(len(states)):
                if (r >> bit) & 1 == 0:
                    q.shard_exchange(states[r], states[r ^ (1 << bit)], local, 0)


class GpuShardBackend:
    """Backend of ``run_rank`` for a shard held as a library State on this
    rank's GPU; halves travel as torch tensors (NCCL)."""

    def __init__(self, shard, fuse_k: int = 0):
        import torch
        self.fuse_k = fuse_k
        # the library's kernels and the collectives share torch's current stream,
        # so a pack is complete before its send and a receive before its unpack
        shard.set_stream(torch.cuda.current_stream())

    def apply(self, shard, gates):
        shard.apply_circuit(gates, fuse_k=self.fuse_k)

    def empty_half(self, shard):
        import torch
        dt = torch.complex128 if shard.dtype == q.C128 else torch.complex64
        return torch.empty(1 << (shard.n - 1), dtype=dt, device="cuda")

    def pack(self, shard, local_qubit, bit):
        buf = self.empty_half(shard)
        q.shard_pack(shard, local_qubit, bit, buf.data_ptr())
        return buf

    def unpack(self, shard, local_qubit, bit, buf):
        q.shard_unpack(shard, local_qubit, bit, buf.data_ptr())


def run_rank(steps, rank: int, shard, backend, dist):
    """Walk a plan as rank `rank` of a torch.distributed group of 2^g ranks:
    apply the gate steps whose rank condition holds, and at each exchange send
    the half of the shard with bit(local) = 1 - bit(rank, rank_bit) to the
    partner rank and put the partner's half in its place."""
    for item in _gate_runs(steps):
        if item[0] == "gates":
            mine = [gt for gt, mask, val in item[1] if (rank & mask) == val]
            if mine:
                backend.apply(shard, mine)
            continue
        _, bit, local = item
        partner = rank ^ (1 << bit)
        half = 1 - ((rank >> bit) & 1)
        out = backend.pack(shard, local, half)
        inc = backend.empty_half(shard)
        reqs = [dist.isend(out, partner), dist.irecv(inc, partner)]
        for r in reqs:
            r.wait()
        backend.unpack(shard, local, half, inc)
