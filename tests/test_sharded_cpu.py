"""The sharded register's host logic on CPU: the exchange planner, the
schedule of ShardedSimulator run on shards backed by the FP64 oracle, and
the same schedule run as two gloo ranks that exchange halves over
torch.distributed (world size 2).  Each is compared with the whole register
on the oracle.  The library's GPU shards are covered by
tests/test_gpu_sharded.py."""
import os
import socket
import sys

import numpy as np
import pytest

import circuitgen as cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleShard:
    """A shard on the oracle: the operations ShardedSimulator asks of one."""

    def __init__(self, n, oracle_mod):
        self.n = n
        self.o = oracle_mod.OracleSim(n)

    def apply(self, m, targets, controls=()):
        self.o.apply(m, list(targets), list(controls))

    def flush(self):
        pass

    def probs_all(self):
        return self.o.probs_all(), self.o.norm2()

    def expect(self, terms):
        return self.o.expect(terms)

    def project(self, qubits, bits, scale, kept_norm2=-1.0):
        idx = np.arange(1 << self.n)
        keep = np.ones(1 << self.n, dtype=bool)
        for q, b in zip(qubits, bits):
            keep &= ((idx >> q) & 1) == b
        self.o.psi[keep] *= scale
        self.o.psi[~keep] = 0.0

    def swap_halves(self, other, qubit):
        a = self.o.psi.reshape(-1, 2, 1 << qubit)
        b = other.o.psi.reshape(-1, 2, 1 << qubit)
        tmp = a[:, 1, :].copy()
        a[:, 1, :] = b[:, 0, :]
        b[:, 0, :] = tmp

    def measure_all(self, u):
        return self.o.measure_all(u)

    def get_amplitudes(self):
        return self.o.psi.copy()

    def set_amplitudes(self, v):
        self.o.psi[:] = v

    def reset(self, basis=0):
        self.o.psi[:] = 0.0
        self.o.psi[basis] = 1.0

    def close(self):
        pass


def mixed_circuit(n, count, seed):
    """Gates on every qubit, global or not: U3, CNOTs both ways, controlled
    U3 with several controls, 2- and 3-qubit random unitaries, Toffoli."""
    rng = np.random.default_rng(seed)
    ops = []
    for k in range(count):
        kind = k % 5
        qs = [int(v) for v in rng.permutation(n)]
        if kind == 0:
            ops.append(cg.op("U3", (qs[0],), (), tuple(rng.uniform(0, 2 * np.pi, 3))))
        elif kind == 1:
            ops.append(cg.op("X", (qs[0],), (qs[1],)))
        elif kind == 2:
            ops.append(cg.op("U3", (qs[0],), (qs[1], qs[2]), tuple(rng.uniform(0, 2 * np.pi, 3))))
        elif kind == 3:
            t = 2 + k % 2
            ops.append(cg.op("MAT", tuple(qs[:t]), (), (cg.random_unitary(1 << t, seed + k),)))
        else:
            ops.append(cg.op("X", (qs[0],), (qs[1], qs[2])))
    return ops


def test_planner_keeps_targets_local_and_is_no_worse_than_lru():
    from paper_1612_08091_gb300.sharded import ExchangePlanner

    rng = np.random.default_rng(3)
    n, g = 12, 3
    needs = [set(int(v) for v in rng.choice(n, size=int(rng.integers(1, 4)), replace=False)) for _ in range(300)]
    p = ExchangePlanner(n, g)
    trace = ExchangePlanner(n, g)
    belady = 0
    for need, steps in zip(needs, p.plan(needs)):
        for G, l in steps:
            assert G >= n - g and l < n - g
            trace.exchange(G, l)
            belady += 1
        assert all(trace.is_local(q) for q in need)
    assert trace.pos == p.pos
    # least-recently-used eviction on the same sequence
    lru = ExchangePlanner(n, g)
    last = {q: -1 for q in range(n)}
    count = 0
    for k, need in enumerate(needs):
        for q in sorted(need):
            if not lru.is_local(q):
                l = min((l for l in range(n - g) if lru.at[l] not in need), key=lambda l: last[lru.at[l]])
                lru.exchange(lru.pos[q], l)
                count += 1
        for q in need:
            last[q] = k
    assert belady <= count, (belady, count)
    # restoring the layout gives the identity
    ex, sw = p.restore()
    assert p.pos == list(range(n)) and p.at == list(range(n))


def test_schedule_reorders_only_commuting_gates(oracle_mod):
    """ExchangePlanner.schedule: every gate once, targets local at their
    step, the order of gates sharing a qubit kept (so the reordered circuit,
    run on the whole register, gives the same state), and on the 32-qubit
    brickwork far fewer exchanges than keeping program order."""
    from paper_1612_08091_gb300.sharded import ExchangePlanner

    n, g = 9, 2
    ops = mixed_circuit(n, 80, seed=5)
    p = ExchangePlanner(n, g)
    trace = ExchangePlanner(n, g)
    order = []
    for step in p.schedule([(op.targets, op.controls) for op in ops]):
        if step[0] == "x":
            trace.exchange(step[1], step[2])
            continue
        k = step[1]
        assert all(trace.is_local(q) for q in ops[k].targets)
        order.append(k)
    assert sorted(order) == list(range(len(ops)))
    for a in range(len(order)):
        for b in range(a + 1, len(order)):
            ka, kb = order[a], order[b]
            qa = set(ops[ka].targets) | set(ops[ka].controls)
            qb = set(ops[kb].targets) | set(ops[kb].controls)
            if qa & qb:
                assert ka < kb
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    re = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(re, [ops[k] for k in order])
    np.testing.assert_allclose(re.psi, ref.psi, atol=1e-12)
    bw = cg.random_u3_brickwork(32, 40, seed=8091)
    steps = ExchangePlanner(32, 1).schedule([(op.targets, op.controls) for op in bw])
    in_order = sum(len(v) for v in ExchangePlanner(32, 1).plan([set(op.targets) for op in bw]))
    ex = sum(1 for st in steps if st[0] == "x")
    assert ex <= 4 < in_order, (ex, in_order)


@pytest.mark.parametrize("g", [1, 2, 3])
def test_sharded_schedule_on_oracle_shards(oracle_mod, g):
    from paper_1612_08091_gb300.sharded import ShardedSimulator

    n = 9
    ops = mixed_circuit(n, 60, seed=100 + g)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    sim = ShardedSimulator(n, global_qubits=g, shard_factory=lambda nl: OracleShard(nl, oracle_mod))
    sim.run(ops)
    sim.flush()
    assert sim.exchanges > 0
    # reads on the permuted layout
    p1, nrm = sim.probs_all()
    np.testing.assert_allclose(p1, ref.probs_all(), atol=1e-12)
    assert abs(nrm - 1.0) <= 1e-12
    rng = np.random.default_rng(g)
    # X factors on at most n - g qubits (they are made local together)
    terms = [(float(rng.normal()), int(rng.choice(n, size=min(n - g, 5), replace=False).tolist() and
                                       sum(1 << int(v) for v in rng.choice(n, size=min(n - g, 4), replace=False))),
              int(rng.integers(0, 1 << n))) for _ in range(12)]
    terms += cg.tfim_terms(n)
    assert abs(sim.expect(terms) - ref.expect(terms)) <= 1e-11
    with pytest.raises(ValueError):
        sim.expect([(1.0, (1 << n) - 1, 0)] if g > 0 else [])
    got = sim.get_amplitudes()
    np.testing.assert_allclose(got, ref.psi, atol=1e-12)
    # measurement of a global and a local qubit, then a full sample
    sim.run(ops[:20])
    oracle_mod.run_ops(ref, ops[:20])
    for q, u in ((n - 1, 0.37), (0, 0.81)):
        b, p = sim.measure(q, u)
        p1 = ref.probs_all()[q]
        assert b == ref.measure(q, u)
        assert abs(p - (p1 if b else 1.0 - p1)) <= 1e-12
        np.testing.assert_allclose(sim.get_amplitudes(), ref.psi, atol=1e-12)
    sim.run(ops[20:40])
    oracle_mod.run_ops(ref, ops[20:40])
    j = sim.measure_all(0.6180339)
    assert j == ref.measure_all(0.6180339)
    np.testing.assert_allclose(sim.get_amplitudes(), ref.psi, atol=1e-12)


# ---------------------------------------------------------------------------
# two gloo ranks, one shard each
# ---------------------------------------------------------------------------
def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, outq):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import circuitgen as cg_
    import oracle
    from paper_1612_08091_gb300 import gates
    from paper_1612_08091_gb300.sharded import (ExchangePlanner, choose_shard, combine_probs, local_terms,
                                                 shard_targets)

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 9
    nl = n - 1
    shard = OracleShard(nl, oracle)
    if rank == 1:
        shard.o.psi[:] = 0.0
    plan = ExchangePlanner(n, 1)

    def exchange(G, l):
        # rank 0 (shard-index bit 0) gives its half with bit l = 1 and takes
        # rank 1's half with bit l = 0
        v = shard.o.psi.reshape(-1, 2, 1 << l)
        mine = torch.from_numpy(np.ascontiguousarray(v[:, 1 - rank, :]).view(np.float64))
        theirs = torch.empty_like(mine)
        if rank == 0:
            dist.send(mine, 1)
            dist.recv(theirs, 1)
        else:
            dist.recv(theirs, 0)
            dist.send(mine, 0)
        v[:, 1 - rank, :] = theirs.numpy().view(np.complex128).reshape(v[:, 1 - rank, :].shape)
        plan.exchange(G, l)

    ops = mixed_circuit(n, 50, seed=77)
    steps = ExchangePlanner(n, 1)
    for st in steps.schedule([(op.targets, op.controls) for op in ops]):
        if st[0] == "x":
            exchange(st[1], st[2])
            continue
        op = ops[st[1]]
        shards, lc = shard_targets(plan, op.controls)
        if rank in shards:
            shard.apply(gates.gate_matrix(op.kind, op.params), [plan.pos[t] for t in op.targets], lc)
    # reductions: all shards' results on every rank, summed in FP64
    p1, nrm = shard.probs_all()
    allp = [torch.zeros(nl + 1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allp, torch.tensor(list(p1) + [nrm], dtype=torch.float64))
    probs, norm = combine_probs(plan, [a[:nl].numpy() for a in allp], [float(a[nl]) for a in allp])
    terms = cg_.tfim_terms(n) + [(0.3, 0, (1 << (n - 1)) | 1), (0.2, 1 << (n - 1), 1 << (n - 1))]
    # terms whose X factors are local now; then each other term after the
    # exchanges that make its X factors local
    e = 0.0
    pending = []
    for t in terms:
        if plan.physical_mask(t[1]) >> nl:
            pending.append(t)
        else:
            e += shard.expect(local_terms(plan, [t], rank))
    for t in pending:
        probe = ExchangePlanner(n, 1)
        probe.pos, probe.at = list(plan.pos), list(plan.at)
        for ex in probe.plan([{q for q in range(n) if (t[1] >> q) & 1}]):
            for G, l in ex:
                exchange(G, l)
        e += shard.expect(local_terms(plan, [t], rank))
    e = torch.tensor([e], dtype=torch.float64)
    dist.all_reduce(e)
    # full-register sample in logical order: restore the layout (exchanges,
    # then SWAP gates inside the shard), then an exclusive scan of the
    # shards' norms
    probe = ExchangePlanner(n, 1)
    probe.pos, probe.at = list(plan.pos), list(plan.at)
    exchanges, local_swaps = probe.restore()
    for G, l in exchanges:
        exchange(G, l)
    for a, b in local_swaps:
        shard.apply(gates.gate_matrix("SWAP", ()), [a, b])
    plan.pos, plan.at = probe.pos, probe.at
    assert plan.pos == list(range(n))
    # the exchanges moved amplitudes between the ranks: gather the norms again
    allw = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allw, torch.tensor([shard.o.norm2()], dtype=torch.float64))
    norms = [float(a[0]) for a in allw]
    s_star, u_loc = choose_shard(norms, 0.42)
    jt = torch.zeros(1, dtype=torch.int64)
    if rank == s_star:
        jt[0] = shard.measure_all(u_loc)
    else:
        shard.project((), (), 0.0)
    dist.broadcast(jt, s_star)
    j_phys = (s_star << nl) | int(jt[0])
    outq.put((rank, probs.tolist(), norm, float(e[0]), plan.logical_index(j_phys), list(plan.pos)))
    dist.destroy_process_group()


def test_two_gloo_ranks_one_shard_each(oracle_mod):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = 9
    ops = mixed_circuit(n, 50, seed=77)
    ref = oracle_mod.OracleSim(n)
    oracle_mod.run_ops(ref, ops)
    terms = cg.tfim_terms(n) + [(0.3, 0, (1 << (n - 1)) | 1), (0.2, 1 << (n - 1), 1 << (n - 1))]
    for rank, probs, norm, e, j, pos in res:
        np.testing.assert_allclose(probs, ref.probs_all(), atol=1e-12)
        assert abs(norm - 1.0) <= 1e-12
        assert pos == res[0][5]
        assert abs(e - ref.expect(terms)) <= 1e-11
    assert res[0][3] == res[1][3]
    assert res[0][4] == res[1][4] == ref.measure_all(0.42)
