"""A register split into shards by its top qubits, with the exchange planner.

The paper's road map (Sec. 5) points to a distributed simulator that splits
the state vector over many nodes.  Here a register of n qubits is split by
its top g physical qubits into 2^g shards of n - g qubits each; shard s holds
the amplitudes whose top g physical bits equal s.  The state is never
gathered:

* a gate whose targets are local (physical position < n - g) runs on every
  shard whose index has all of the gate's global control bits set, with the
  local controls passed on;
* a target held in the shard index ("global" qubit) is first exchanged with a
  local position: for shard pairs (s, s | 2^j) the halves where local bit l
  and global bit j differ trade places (``sim_swap_halves``), and the two
  logical qubits swap physical positions.  The exchange planner chooses the
  local position to give up by Belady's rule: the one whose logical qubit is
  next needed as a target furthest in the future;
* reductions are FP64 sums of the shards' partial results; a measurement
  decides its outcome on the summed probabilities and then projects every
  shard with the common scale 1/sqrt(p) (``sim_project``); a full-register
  sample picks the shard by an exclusive scan of the shards' norms and
  samples inside it.

``ExchangePlanner`` and the combination helpers are host logic with no
arithmetic on amplitudes; ``ShardedSimulator`` runs the shards as handles of
libqsim on one GPU (every device step in the library's kernels).  On a
machine with one GPU per shard the same schedule would move the exchanged
halves between devices; here all shards share one device.
"""
import bisect
import heapq

import numpy as np

from . import gates as _gates
from .qsim import Simulator


class ExchangePlanner:
    """Layout of logical qubits on physical positions and the exchanges that
    make gate targets local.  Positions 0..n-g-1 are local (bits of the
    index inside a shard), n-g..n-1 global (bits of the shard index)."""

    def __init__(self, n, g):
        if g < 0 or g >= n:
            raise ValueError("need 0 <= g < n")
        self.n, self.g, self.nl = int(n), int(g), int(n) - int(g)
        self.pos = list(range(self.n))  # logical qubit -> physical position
        self.at = list(range(self.n))   # physical position -> logical qubit

    def reset(self):
        self.pos = list(range(self.n))
        self.at = list(range(self.n))

    def is_local(self, q):
        return self.pos[q] < self.nl

    def exchange(self, G, l):
        """Record that global position G and local position l traded contents."""
        a, b = self.at[G], self.at[l]
        self.at[G], self.at[l] = b, a
        self.pos[a], self.pos[b] = l, G

    def plan(self, needs):
        """needs[k]: the logical qubits that must be local at step k.  Returns,
        per step, the exchanges (global position, local position) to make
        before it, in order, and updates the layout as they are made."""
        for k, need in enumerate(needs):
            if len(need) > self.nl:
                raise ValueError("step %d needs %d local qubits, the shards have %d" % (k, len(need), self.nl))
        uses = [[] for _ in range(self.n)]
        for k, need in enumerate(needs):
            for q in need:
                uses[q].append(k)
        out = []
        for k, need in enumerate(needs):
            steps = []
            for q in sorted(need):
                if self.is_local(q):
                    continue
                best, best_next = None, -1
                for l in range(self.nl):
                    v = self.at[l]
                    if v in need:
                        continue
                    u = uses[v]
                    i = bisect.bisect_right(u, k)
                    nxt = u[i] if i < len(u) else len(needs) + 1
                    if nxt > best_next:
                        best, best_next = l, nxt
                G = self.pos[q]
                self.exchange(G, best)
                steps.append((G, best))
            out.append(steps)
        return out

    def schedule(self, gates):
        """Order a list of gates ((targets, controls) in logical qubits) for
        execution with as few exchanges as the greedy rule finds, keeping
        the order of any two gates that share a qubit.  Gates whose targets
        are local run as soon as every earlier gate on their qubits has run;
        only when every remaining ready gate needs a global target is an
        exchange made: the global target of the earliest such gate comes in,
        and the local position given up is the one whose logical qubit is
        next needed as a target furthest ahead in program order.  Long runs
        of gates then sit between exchanges, and the shards fuse them into
        blocks.  Returns a list of ("x", G, l) and ("g", index) steps and
        leaves the layout as after the last step."""
        ng = len(gates)
        for k, (t, _) in enumerate(gates):
            if len(t) > self.nl:
                raise ValueError("gate %d needs %d local qubits, the shards have %d" % (k, len(t), self.nl))
        per_q = [[] for _ in range(self.n)]  # program-order gate indices on each qubit
        tuses = [[] for _ in range(self.n)]  # ... where the qubit is a target
        for k, (t, c) in enumerate(gates):
            for q in set(t) | set(c):
                per_q[q].append(k)
            for q in t:
                tuses[q].append(k)
        head = [0] * self.n  # next pending position in per_q[q]
        tnext = [0] * self.n  # next pending position in tuses[q]
        done = [False] * ng

        def is_ready(k):
            t, c = gates[k]
            return all(per_q[q][head[q]] == k for q in set(t) | set(c))

        out = []
        heap = sorted({per_q[q][0] for q in range(self.n) if per_q[q] and is_ready(per_q[q][0])})
        waiting = []  # ready gates blocked on a global target
        remaining = ng
        while remaining:
            while heap:
                k = heapq.heappop(heap)
                t, c = gates[k]
                if not all(self.is_local(q) for q in t):
                    waiting.append(k)
                    continue
                out.append(("g", k))
                done[k] = True
                remaining -= 1
                for q in set(t) | set(c):
                    head[q] += 1
                    if head[q] < len(per_q[q]):
                        nk = per_q[q][head[q]]
                        if is_ready(nk):
                            heapq.heappush(heap, nk)
                for q in t:
                    tnext[q] += 1
            if not remaining:
                break
            # every ready gate waits for a global target: bring in the
            # earliest one's
            waiting = sorted(set(w for w in waiting if not done[w]))
            k = waiting[0]
            t, _ = gates[k]
            q = next(q for q in t if not self.is_local(q))
            best, best_next = None, -1
            for l in range(self.nl):
                v = self.at[l]
                if v in t:
                    continue
                u = tuses[v]
                nxt = u[tnext[v]] if tnext[v] < len(u) else ng + 1
                if nxt > best_next:
                    best, best_next = l, nxt
            G = self.pos[q]
            self.exchange(G, best)
            out.append(("x", G, best))
            for w in waiting:
                heapq.heappush(heap, w)
            waiting = []
        return out

    def restore(self):
        """Exchanges (G, l) and then local position swaps (a, b) that bring
        every logical qubit back to its own position."""
        exchanges = []
        for G in range(self.nl, self.n):
            if self.at[G] == G:
                continue
            p = self.pos[G]
            if p >= self.nl:  # held by another global position: route through a local one
                l = 0
                self.exchange(p, l)
                exchanges.append((p, l))
                p = l
            self.exchange(G, p)
            exchanges.append((G, p))
        local_swaps = []
        for l in range(self.nl):
            if self.at[l] != l:
                p = self.pos[l]
                a, b = self.at[l], self.at[p]
                self.at[l], self.at[p] = b, a
                self.pos[a], self.pos[b] = p, l
                local_swaps.append((l, p))
        return exchanges, local_swaps

    # -- mapping ---------------------------------------------------------------
    def split_controls(self, controls):
        """Physical local controls and the mask of required shard-index bits."""
        local, gmask = [], 0
        for c in controls:
            p = self.pos[c]
            if p < self.nl:
                local.append(p)
            else:
                gmask |= 1 << (p - self.nl)
        return local, gmask

    def physical_mask(self, mask):
        out = 0
        q = 0
        while mask:
            if mask & 1:
                out |= 1 << self.pos[q]
            mask >>= 1
            q += 1
        return out

    def logical_index(self, phys):
        """Logical basis index of a physical index."""
        out = 0
        for q in range(self.n):
            out |= ((phys >> self.pos[q]) & 1) << q
        return out


def shard_targets(planner, controls):
    """Indices of the shards a gate with these logical controls runs on, and
    its physical local controls."""
    local, gmask = planner.split_controls(controls)
    return [s for s in range(1 << planner.g) if (s & gmask) == gmask], local


def combine_probs(planner, shard_p1, shard_norm):
    """P(logical qubit q = 1) for all q and the norm, from each shard's
    P(local bit = 1) and norm (FP64 sums)."""
    nl = planner.nl
    phys = np.zeros(planner.n)
    for s, (p1, nrm) in enumerate(zip(shard_p1, shard_norm)):
        phys[:nl] += np.asarray(p1, dtype=np.float64)
        for j in range(planner.g):
            if (s >> j) & 1:
                phys[nl + j] += nrm
    return np.array([phys[planner.pos[q]] for q in range(planner.n)]), float(sum(shard_norm))


def choose_shard(shard_norm, u):
    """Full-register sampling over shards: the shard s whose cumulative norm
    interval (exclusive scan) holds u * total, and the draw to use inside it,
    so that the local cumulative sum crosses u * total where the global one
    does."""
    total = float(sum(shard_norm))
    target = u * total
    prefix = 0.0
    last = None
    for s, w in enumerate(shard_norm):
        if w > 0.0:
            last = s
            if prefix + w > target:
                return s, min(max((target - prefix) / w, 0.0), np.nextafter(1.0, 0.0))
        prefix += w
    if last is None:
        raise ValueError("all shards are zero")
    return last, np.nextafter(1.0, 0.0)


def local_terms(planner, terms, s):
    """A Pauli sum as seen by shard s: each term's X / Z masks on physical
    local positions, with the sign of its Z factors on global positions.
    Every X factor must be on a local position."""
    nl = planner.nl
    low = (1 << nl) - 1
    out = []
    for c, x, z in terms:
        px, pz = planner.physical_mask(int(x)), planner.physical_mask(int(z))
        if px >> nl:
            raise ValueError("X factor on a global qubit")
        sign = -1.0 if bin((pz >> nl) & s).count("1") & 1 else 1.0
        out.append((sign * float(c), px & low, pz & low))
    return out


class ShardedSimulator:
    """An n-qubit register held as 2^g shards of n - g qubits on one GPU.
    Gates are queued lazily; on flush the exchange planner makes every
    gate's targets local and the shards run their own queues (and fusion)."""

    def __init__(self, n, global_qubits=1, precision="c128", fusion="none", kmax=6, shard_factory=None, **kw):
        """shard_factory(n_local) makes one shard; by default a libqsim
        Simulator handle on the current GPU with the given precision, fusion
        and options.  (The schedule itself is device-independent, which is how
        the tests check it without a GPU.)"""
        self.n = int(n)
        self.g = int(global_qubits)
        self.planner = ExchangePlanner(self.n, self.g)
        self.nl = self.planner.nl
        if shard_factory is None:
            def shard_factory(nl):
                return Simulator(nl, precision=precision, fusion=fusion, kmax=kmax, **kw)
        self.shards = [shard_factory(self.nl) for _ in range(1 << self.g)]
        self.queue = []
        self.exchanges = 0
        for sh in self.shards[1:]:
            sh.project((), (), 0.0)

    # -- plumbing ----------------------------------------------------------------
    def close(self):
        for sh in self.shards:
            sh.close()
        self.shards = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _exchange(self, G, l):
        j = G - self.nl
        for s in range(1 << self.g):
            if not (s >> j) & 1:
                self.shards[s].swap_halves(self.shards[s | (1 << j)], l)
        self.exchanges += 1

    def _make_local(self, needs):
        for steps in self.planner.plan(needs):
            for G, l in steps:
                self._exchange(G, l)

    # -- gates -------------------------------------------------------------------
    def apply(self, matrix, targets, controls=()):
        self.queue.append((np.ascontiguousarray(matrix, dtype=np.complex128), tuple(int(t) for t in targets),
                           tuple(int(c) for c in controls)))

    def apply_op(self, op):
        self.apply(_gates.gate_matrix(op.kind, op.params), op.targets, op.controls)

    def run(self, ops):
        for op in ops:
            self.apply_op(op)

    def flush(self):
        q, self.queue = self.queue, []
        if not q:
            return
        plan = self.planner
        # replay the schedule step by step so each gate sees its layout
        sched = ExchangePlanner(self.n, self.g)
        sched.pos, sched.at = list(plan.pos), list(plan.at)
        for step in sched.schedule([(t, c) for _, t, c in q]):
            if step[0] == "x":
                self._exchange(step[1], step[2])
                plan.exchange(step[1], step[2])
                continue
            m, t, c = q[step[1]]
            pt = [plan.pos[x] for x in t]
            shards, lc = shard_targets(plan, c)
            for s in shards:
                self.shards[s].apply(m, pt, lc)
        for sh in self.shards:
            sh.flush()

    # -- reads -------------------------------------------------------------------
    def _shard_probs(self):
        self.flush()
        res = [sh.probs_all() for sh in self.shards]
        return [r[0] for r in res], [r[1] for r in res]

    def probs_all(self):
        p1s, norms = self._shard_probs()
        return combine_probs(self.planner, p1s, norms)

    def prob(self, qubit):
        return float(self.probs_all()[0][qubit])

    def expect(self, terms):
        self.flush()
        terms = [(float(c), int(x), int(z)) for c, x, z in terms]
        total = 0.0
        pending = []
        ready = []
        for t in terms:
            xq = {q for q in range(self.n) if (t[1] >> q) & 1}
            if len(xq) > self.nl:
                raise ValueError("a term with X or Y factors on %d qubits needs them local together; the shards "
                                 "have %d local qubits" % (len(xq), self.nl))
            (ready if all(self.planner.is_local(q) for q in xq) else pending).append((t, xq))
        groups = [[t for t, _ in ready]] + [[t] for t, _ in pending]
        needs = [set()] + [xq for _, xq in pending]
        for grp, need in zip(groups, needs):
            if need:
                self._make_local([need])
            if not grp:
                continue
            for s, sh in enumerate(self.shards):
                total += sh.expect(local_terms(self.planner, grp, s))
        return total

    def measure(self, qubit, u):
        p1s, norms = self._shard_probs()
        p1, norm = combine_probs(self.planner, p1s, norms)
        P1 = p1[qubit]
        P0 = norm - P1
        b = 0 if u * norm < P0 else 1
        pb = P1 if b else P0
        if not pb > 0.0:
            raise ValueError("measured outcome has probability 0")
        scale = 1.0 / np.sqrt(pb)
        p = self.planner.pos[qubit]
        for s, sh in enumerate(self.shards):
            if p < self.nl:
                kept = p1s[s][p] if b else norms[s] - p1s[s][p]
                sh.project((p,), (b,), scale, max(kept, 0.0))
            else:
                keep = ((s >> (p - self.nl)) & 1) == b
                sh.project((), (), scale if keep else 0.0, norms[s])
        return b, pb / norm

    def measure_all(self, u):
        # the cumulative sums run over logical basis order, which is the
        # shards' physical order only in the identity layout
        self.restore_layout()
        _, norms = self._shard_probs()
        s_star, u_local = choose_shard(norms, u)
        j = self.shards[s_star].measure_all(u_local)
        for s, sh in enumerate(self.shards):
            if s != s_star:
                sh.project((), (), 0.0)
        return self.planner.logical_index((s_star << self.nl) | j)

    # -- state ---------------------------------------------------------------------
    def restore_layout(self):
        """Bring every logical qubit back to its own position (device work:
        exchanges, then SWAP gates inside the shards)."""
        self.flush()
        probe = ExchangePlanner(self.n, self.g)
        probe.pos, probe.at = list(self.planner.pos), list(self.planner.at)
        exchanges, local_swaps = probe.restore()
        for G, l in exchanges:
            self._exchange(G, l)
        swap = _gates.gate_matrix("SWAP", ())
        for a, b in local_swaps:
            for sh in self.shards:
                sh.apply(swap, (a, b))
        for sh in self.shards:
            sh.flush()
        self.planner.pos, self.planner.at = probe.pos, probe.at

    def get_amplitudes(self):
        self.restore_layout()
        return np.concatenate([sh.get_amplitudes() for sh in self.shards])

    def set_amplitudes(self, values):
        v = np.ascontiguousarray(values, dtype=np.complex128)
        if v.shape != (1 << self.n,):
            raise ValueError("expected %d amplitudes" % (1 << self.n))
        self.queue = []
        self.planner.reset()
        L = 1 << self.nl
        for s, sh in enumerate(self.shards):
            sh.set_amplitudes(v[s * L:(s + 1) * L])

    def reset(self, basis=0):
        self.queue = []
        self.planner.reset()
        s_star = int(basis) >> self.nl
        for s, sh in enumerate(self.shards):
            sh.reset(int(basis) & ((1 << self.nl) - 1))
            if s != s_star:
                sh.project((), (), 0.0)
