"""One state over 2^g shards, on CPU: the library's exchange plan
(qc_shard_plan, host only) walked with the FP64 oracle on each shard.

The whole-register result must equal the oracle run of the unsharded circuit
(Eq. (1) gate by gate).  In-process cases cover 1..3 global qubits with gates
whose targets or controls sit on global qubits (control states 0 and 1),
2- and 3-qubit blocks with every target global, SWAP gates (relabelled, no
data moved) and the QFT.  The multi-process cases run the same protocol as
2 and 4 gloo ranks, each holding one shard and trading halves with
torch.distributed send/recv.
"""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_00123_gb300 import circuits as C
from paper_2303_00123_gb300.circuits import Gate


def _q():
    from paper_2303_00123_gb300 import qcgb300
    return qcgb300


class OracleBackend:
    """A shard as a numpy vector; gates by the oracle; halves as torch CPU tensors."""

    def __init__(self, nloc):
        self.nloc = nloc

    def apply(self, shard, gates):
        for gt in gates:
            O.apply_gate(shard, self.nloc, gt)

    @staticmethod
    def _idx(nloc, local, bit):
        pb = nloc - 1 - local
        j = np.arange(1 << (nloc - 1), dtype=np.int64)
        lo = j & ((1 << pb) - 1)
        return ((j ^ lo) << 1) | lo | (bit << pb)

    def empty_half(self, shard):
        import torch
        return torch.empty(1 << (self.nloc - 1), dtype=torch.complex128)

    def pack(self, shard, local, bit):
        import torch
        return torch.from_numpy(shard[self._idx(self.nloc, local, bit)].copy())

    def unpack(self, shard, local, bit, buf):
        shard[self._idx(self.nloc, local, bit)] = buf.numpy()


def emulate(n, g, steps, psi0):
    """All shards in one process (the exchange done directly)."""
    nloc = n - g
    shards = [psi0[r << nloc:(r + 1) << nloc].copy() for r in range(1 << g)]
    be = OracleBackend(nloc)
    for st in steps:
        if st[0] == "gate":
            _, gt, mask, val = st
            for r in range(1 << g):
                if (r & mask) == val:
                    O.apply_gate(shards[r], nloc, gt)
        else:
            _, bit, local = st
            for r in range(1 << g):
                if (r >> bit) & 1 == 0:
                    p = r ^ (1 << bit)
                    ia, ib = be._idx(nloc, local, 1), be._idx(nloc, local, 0)
                    shards[r][ia], shards[p][ib] = shards[p][ib].copy(), shards[r][ia].copy()
    return np.concatenate(shards)


def wide_blocks(n, rng, count):
    out = []
    for _ in range(count):
        k = int(rng.integers(2, 4))
        qs = [int(v) for v in rng.choice(n, size=k, replace=False)]
        out.append(Gate("UK" if k > 2 else "U4", tuple(qs), matrix=C.haar_unitary(rng, 1 << k)))
    return out


@pytest.mark.parametrize("g", [1, 2, 3])
@pytest.mark.parametrize("n", [7, 9])
def test_plan_reproduces_the_circuit(n, g):
    q = _q()
    rng = np.random.default_rng(10 * n + g)
    gates = C.random_mix(n, 80, seed=n + g) + wide_blocks(n, rng, 10) + C.qft(n)
    # every global qubit as a target together with the others, and as a control in both states
    gates += [Gate("UK", tuple(range(g)) + ((g,) if g < 3 else ()), matrix=C.haar_unitary(rng, 1 << (g + (g < 3))))]
    gates += [Gate("U", (n - 1,), controls=(0,), cstates=(0,), matrix=C.haar_unitary(rng, 2)),
              Gate("X", (n - 2,), controls=(n - 1, g - 1), cstates=(1, 0)),
              Gate("Y", (0,), controls=(n - 1,), cstates=(1,)), Gate("SWAP", (0, n - 1)),
              Gate("U4", (n - 2, 0), matrix=C.haar_unitary(rng, 4))]
    steps = q.shard_plan(n, g, gates)
    psi0 = C.random_state(n, 5)
    got = emulate(n, g, steps, psi0)
    ref = O.run_circuit(n, gates, psi0)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    # exchanges happened, and every exchange names a valid rank bit and local qubit
    ex = [s for s in steps if s[0] == "exchange"]
    assert ex and all(0 <= s[1] < g and 0 <= s[2] < n - g for s in ex)


def test_swaps_move_no_data_and_local_gates_need_no_exchange():
    q = _q()
    n, g = 8, 2
    local = [Gate("H", (q_,)) for q_ in range(g, n)] + [Gate("X", (5,), controls=(0, 1), cstates=(1, 0))]
    steps = q.shard_plan(n, g, local)
    assert all(s[0] == "gate" for s in steps)
    ctl = steps[-1]
    assert ctl[2] == 0b11 and ctl[3] == 0b10          # controls on qubits 0, 1 -> rank bits 1, 0
    swaps = [Gate("SWAP", (0, 3)), Gate("SWAP", (1, 6)), Gate("SWAP", (0, 3)), Gate("SWAP", (1, 6))]
    assert q.shard_plan(n, g, swaps) == []             # relabelled there and back: nothing to do
    steps = q.shard_plan(n, g, swaps[:1])              # one SWAP: restoring the layout is one exchange
    assert [s[0] for s in steps] == ["exchange"]
    psi0 = C.random_state(n, 6)
    np.testing.assert_allclose(emulate(n, g, steps, psi0), O.run_circuit(n, swaps[:1], psi0), atol=0)


def test_plan_rejects_what_does_not_fit():
    q = _q()
    with pytest.raises(q.QCError):
        q.shard_plan(4, 4, [Gate("H", (0,))])          # no local qubit left
    with pytest.raises(q.QCError):
        q.shard_plan(6, 3, [Gate("UK", (0, 1, 2, 3), matrix=np.eye(16))])   # 4 targets, 3 local qubits
    with pytest.raises(q.QCError):
        q.shard_plan(6, 2, [Gate("H", (6,))])          # qubit out of range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_worker(rank, world, port, n, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2303_00123_gb300 import shard
    g = world.bit_length() - 1
    gates = C.random_mix(n, 60, seed=11) + C.qft(n) + C.brickwork(n, 3, seed=12)
    steps = _q().shard_plan(n, g, gates)
    nloc = n - g
    psi0 = C.random_state(n, 13)
    mine = psi0[rank << nloc:(rank + 1) << nloc].copy()
    shard.run_rank(steps, rank, mine, OracleBackend(nloc), dist)
    out.put((rank, mine))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_exchange_halves(world):
    import torch.multiprocessing as mp
    n = 8
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker, args=(r, world, port, n, qu)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(qu.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([res[r] for r in range(world)])
    gates = C.random_mix(n, 60, seed=11) + C.qft(n) + C.brickwork(n, 3, seed=12)
    ref = O.run_circuit(n, gates, C.random_state(n, 13))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
