"""Gate DAG and acyclic part builders of the oracle (test infrastructure).

Written from Sec. IV of the paper:

* Sec. IV-A: gates are DAG vertices, qubit wires are edges; every qubit has
  an artificial entry and exit vertex; the working set L(V_i) of a part is the
  number of distinct qubits its gates use; an acyclic k-way partition has
  disjoint, exhaustive, non-empty parts with L <= L_m and an acyclic part
  graph; gates of a part run in their original relative order.
* Sec. IV-B: Nat (cut-off along the circuit order), DFS (the same cut-off
  along several random DFS topological orders, keep the fewest parts) and
  dagP (recursive bisection until L <= L_m, then a merge phase on the part
  graph that keeps it acyclic and L <= L_m). L of a convex part equals the
  number of wire edges entering it plus the entry vertices inside it.

Where Sec. IV-B leaves details open (it defers the builders' internals to
external work), these readings are used:

* Nat: gate g joins the open part iff L(part + g) <= k, else the part is
  closed and g opens the next one.
* DFS: trial r uses SplitMix64(seed XOR r*0x9E3779B97F4A7C15); the order is a
  LIFO Kahn traversal: the source gates are shuffled (Fisher-Yates) onto a
  stack; each popped gate is emitted and its successors whose in-degree
  reaches zero (in operand order) are shuffled and pushed. 16 trials by
  default; fewest parts wins, ties to the lowest r.
* dagP: bisection cut = prefix of the part's ascending gate order minimising
  L(V1) + L(V2) among cuts whose larger side has at most floor(3|P|/4)
  gates (imbalance ratio 1.5 of the average side), ties by |2c - |P|| then
  smaller c; refinement = best single move with positive gain in
  L(V1) + L(V2) keeping V1 a down-set, both sides non-empty and within the
  same size cap, ties by smaller gate id, at most 4|P| moves; recurse on V1
  then V2; merge phase = repeatedly merge the pair with L(a u b) <= k, no path
  of length >= 2 between them, most shared qubits, ties by the smaller
  (min gate of the pair, max gate of the pair) key.
* Schedule: Kahn order of the part graph with a min-heap keyed by each
  part's smallest gate index; parts are renumbered 0..P-1 in that order.

Beyond the paper: ``beam`` states the repository's beam-search builder from
its definition (see its docstring) so that the C++ builder's partitions are
checked bit for bit, and ``brute_force_min_parts`` gives the optimum on tiny
DAGs.

Gates are ``(name, qubits, theta)`` tuples (``synth``).
"""
from __future__ import annotations

import heapq

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


class PartitionError(ValueError):
    pass


class _SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014), this module's own copy."""

    def __init__(self, seed):
        self.s = seed & MASK64

    def next(self):
        self.s = (self.s + GOLDEN) & MASK64
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def shuffle(self, a):
        for i in range(len(a) - 1, 0, -1):
            j = self.next() % (i + 1)
            a[i], a[j] = a[j], a[i]


class Dag:
    """Gate DAG of Sec. IV-A. preds/succs list distinct neighbour gates in
    operand order; wire_prev[g][j] is the gate before g on its j-th operand
    (-1 = the qubit's entry vertex)."""

    def __init__(self, gates, n):
        self.n = n
        self.G = len(gates)
        self.qubits = [tuple(g[1]) for g in gates]
        self.qmask = []
        last = [-1] * n
        self.wire_prev = []
        self.preds = []
        self.succs = [[] for _ in range(self.G)]
        for g, qs in enumerate(self.qubits):
            m = 0
            wp = []
            for q in qs:
                if not (0 <= q < n):
                    raise PartitionError(f"gate {g}: qubit {q} out of range")
                if (m >> q) & 1:
                    raise PartitionError(f"gate {g}: repeated qubit {q}")
                m |= 1 << q
                wp.append(last[q])
            self.qmask.append(m)
            self.wire_prev.append(wp)
            pr = []
            for p in wp:
                if p >= 0 and p not in pr:
                    pr.append(p)
            self.preds.append(pr)
            for q in qs:
                last[q] = g
        for g in range(self.G):
            for p in self.preds[g]:
                self.succs[p].append(g)
        # succs were appended in increasing g; reorder to operand order of g
        for p in range(self.G):
            seen = []
            # the successor on each operand wire of p, in operand order
            for q in self.qubits[p]:
                nxt = self._next_on_wire(p, q)
                if nxt >= 0 and nxt not in seen:
                    seen.append(nxt)
            self.succs[p] = seen
        self.first_gate = [-1] * n
        for g, qs in enumerate(self.qubits):
            for q in qs:
                if self.first_gate[q] < 0:
                    self.first_gate[q] = g

    def _next_on_wire(self, g, q):
        if not hasattr(self, "_next_cache"):
            nxt = {}
            lastg = {}
            for h, qs in enumerate(self.qubits):
                for qq in qs:
                    if qq in lastg:
                        nxt[(lastg[qq], qq)] = h
                    lastg[qq] = h
            self._next_cache = nxt
        return self._next_cache.get((g, q), -1)


def working_set(dag: Dag, gate_ids) -> int:
    """L(V_i): number of distinct qubits used by the gates (Sec. IV-A)."""
    m = 0
    for g in gate_ids:
        m |= dag.qmask[g]
    return bin(m).count("1")


def working_set_by_edges(dag: Dag, gate_ids) -> int:
    """L of a convex part counted as in Sec. IV-B: wire edges entering the part
    from a gate outside it plus entry vertices whose first gate is inside."""
    s = set(gate_ids)
    cnt = 0
    for g in s:
        for j, p in enumerate(dag.wire_prev[g]):
            if p < 0:
                cnt += 1          # entry vertex of this qubit belongs to the part
            elif p not in s:
                cnt += 1          # in-edge from another part
    return cnt


def _check_arity(dag: Dag, k: int):
    if k < 1:
        raise PartitionError("k must be >= 1")
    for g in range(dag.G):
        if len(dag.qubits[g]) > k:
            raise PartitionError(f"gate {g} has arity {len(dag.qubits[g])} > k={k}")


def cut_order(dag: Dag, order, k: int):
    """Cut-off along a topological order (Nat rule): list of parts, each a
    list of gate ids in the order visited."""
    parts = []
    cur = []
    m = 0
    for g in order:
        gm = dag.qmask[g]
        if cur and bin(m | gm).count("1") > k:
            parts.append(cur)
            cur = []
            m = 0
        cur.append(g)
        m |= gm
    if cur:
        parts.append(cur)
    return parts


def _parts_to_pog(G, parts):
    pog = [-1] * G
    for i, p in enumerate(parts):
        for g in p:
            pog[g] = i
    return pog


def nat(gates, n, k):
    dag = Dag(gates, n)
    _check_arity(dag, k)
    parts = cut_order(dag, range(dag.G), k)
    return schedule(dag, _parts_to_pog(dag.G, parts))


def dfs_order(dag: Dag, rng: _SplitMix64):
    indeg = [len(p) for p in dag.preds]
    stack = [g for g in range(dag.G) if indeg[g] == 0]
    rng.shuffle(stack)
    order = []
    while stack:
        g = stack.pop()
        order.append(g)
        newly = []
        for s in dag.succs[g]:
            indeg[s] -= 1
            if indeg[s] == 0:
                newly.append(s)
        rng.shuffle(newly)
        stack.extend(newly)
    return order


def dfs(gates, n, k, seed=0, trials=16):
    dag = Dag(gates, n)
    _check_arity(dag, k)
    best = None
    for r in range(trials):
        rng = _SplitMix64(seed ^ ((r * GOLDEN) & MASK64))
        order = dfs_order(dag, rng)
        parts = cut_order(dag, order, k)
        if best is None or len(parts) < len(best):
            best = parts
    if best is None:
        best = []
    return schedule(dag, _parts_to_pog(dag.G, best))


# ---------------------------------------------------------------- dagP ----

def _topo_units(succ, pred, live, mg):
    """Kahn order of the units with a min-heap keyed by each unit's smallest gate."""
    indeg = {u: 0 for u in live}
    for u in live:
        for v in succ[u]:
            indeg[v] += 1
    h = [(mg[u], u) for u in live if indeg[u] == 0]
    heapq.heapify(h)
    out = []
    while h:
        _, u = heapq.heappop(h)
        out.append(u)
        for v in succ[u]:
            indeg[v] -= 1
            if indeg[v] == 0:
                heapq.heappush(h, (mg[v], v))
    if len(out) != len(live):
        raise PartitionError("part graph has a cycle")
    return out


class _Units:
    """Groups of gates (units) with their part graph, used by all dagP phases.

    Each unit has its sorted gate list, qubit mask, smallest gate (mg), direct
    successor / predecessor units and ``reach``: the set of units reachable
    through one or more edges, as an int bitset over unit ids."""

    def __init__(self, dag: Dag, groups):
        self.dag = dag
        self.gates, self.qm, self.mg = {}, {}, {}
        unit_of = [0] * dag.G
        for i, grp in enumerate(groups):
            gl = sorted(grp)
            self.gates[i] = gl
            m = 0
            for g in gl:
                m |= dag.qmask[g]
                unit_of[g] = i
            self.qm[i] = m
            self.mg[i] = gl[0]
        self.next_id = len(groups)
        self.succ = {i: set() for i in self.gates}
        self.pred = {i: set() for i in self.gates}
        for g in range(dag.G):
            a = unit_of[g]
            for t in dag.succs[g]:
                b = unit_of[t]
                if b != a:
                    self.succ[a].add(b)
                    self.pred[b].add(a)
        order = _topo_units(self.succ, self.pred, list(self.gates), self.mg)
        self.reach = {}
        for u in reversed(order):
            r = 0
            for v in self.succ[u]:
                r |= (1 << v) | self.reach[v]
            self.reach[u] = r

    def long_path(self, a, b):
        """True iff a path of length >= 2 joins a and b (either direction)."""
        for c in self.succ[a]:
            if (self.reach[c] >> b) & 1:
                return True
        for c in self.succ[b]:
            if (self.reach[c] >> a) & 1:
                return True
        return False

    def merge(self, a, b):
        c = self.next_id
        self.next_id += 1
        mab = (1 << a) | (1 << b)
        self.gates[c] = sorted(self.gates.pop(a) + self.gates.pop(b))
        self.qm[c] = self.qm.pop(a) | self.qm.pop(b)
        self.mg[c] = min(self.mg.pop(a), self.mg.pop(b))
        sc = (self.succ.pop(a) | self.succ.pop(b)) - {a, b}
        pc = (self.pred.pop(a) | self.pred.pop(b)) - {a, b}
        self.succ[c], self.pred[c] = sc, pc
        for x in sc:
            self.pred[x] -= {a, b}
            self.pred[x].add(c)
        for x in pc:
            self.succ[x] -= {a, b}
            self.succ[x].add(c)
        rc = (self.reach.pop(a) | self.reach.pop(b)) & ~mab
        for x in self.reach:
            r = self.reach[x]
            if r & mab:
                self.reach[x] = (r & ~mab) | (1 << c) | rc
        self.reach[c] = rc
        return c

    def merge_loop(self, k, zero_shared):
        """Repeatedly merge the valid pair with the smallest key
        (-shared qubits, smaller min gate, larger min gate); valid = merged
        L <= k and no path of length >= 2 between the two units. With
        zero_shared False only pairs sharing a qubit are candidates."""
        heap = []
        byq = [set() for _ in range(self.dag.n)]
        for u, m in self.qm.items():
            q = 0
            while m:
                if m & 1:
                    byq[q].add(u)
                m >>= 1
                q += 1

        def key_push(a, b):
            qa, qb = self.qm[a], self.qm[b]
            if bin(qa | qb).count("1") > k:
                return
            ma, mb = self.mg[a], self.mg[b]
            m1, m2 = (ma, mb) if ma < mb else (mb, ma)
            heapq.heappush(heap, (-bin(qa & qb).count("1"), m1, m2, a, b))

        def sharing(u):
            out = set()
            m = self.qm[u]
            q = 0
            while m:
                if m & 1:
                    out |= byq[q]
                m >>= 1
                q += 1
            out.discard(u)
            return out

        for u in sorted(self.qm):
            for v in sharing(u):
                if v > u:
                    key_push(u, v)
        zero_done = False
        while True:
            if not heap:
                if not zero_shared or zero_done:
                    break
                zero_done = True
                live = sorted(self.qm)
                for i in range(len(live)):
                    for j in range(i + 1, len(live)):
                        if not (self.qm[live[i]] & self.qm[live[j]]):
                            key_push(live[i], live[j])
                if not heap:
                    break
                continue
            _, _, _, a, b = heapq.heappop(heap)
            if a not in self.qm or b not in self.qm:
                continue
            if self.long_path(a, b):
                continue
            ma, mb = self.qm[a], self.qm[b]
            c = self.merge(a, b)
            q = 0
            m = ma | mb
            while m:
                if m & 1:
                    byq[q].discard(a)
                    byq[q].discard(b)
                    byq[q].add(c)
                m >>= 1
                q += 1
            if zero_done:
                for v in sorted(self.qm):
                    if v != c:
                        key_push(v, c)
            else:
                for v in sorted(sharing(c)):
                    key_push(v, c)


def _side_cap(W):
    """Largest allowed side weight of a bisection of total weight W:
    imbalance ratio 1.5 of the average side, floor(1.5 * W / 2)."""
    return (3 * W) // 4


def _bisect_units(U: _Units, seq, k):
    """Prefix cut of a topologically ordered unit sequence minimising
    L(V1) + L(V2); side weights (gate counts) within the cap when any cut
    allows it; ties by |2 w(V1) - W| then smaller c."""
    m = len(seq)
    w = [len(U.gates[u]) for u in seq]
    W = sum(w)
    pre = [0] * (m + 1)
    prew = [0] * (m + 1)
    mask = 0
    for i in range(m):
        mask |= U.qm[seq[i]]
        pre[i + 1] = bin(mask).count("1")
        prew[i + 1] = prew[i] + w[i]
    suf = [0] * (m + 1)
    mask = 0
    for i in range(m - 1, -1, -1):
        mask |= U.qm[seq[i]]
        suf[i] = bin(mask).count("1")
    cap = _side_cap(W)
    best = None
    for balanced in (True, False):
        for c in range(1, m):
            if balanced and max(prew[c], W - prew[c]) > cap:
                continue
            key = (pre[c] + suf[c], abs(2 * prew[c] - W), c)
            if best is None or key < best:
                best = key
        if best is not None:
            break
    c = best[2]
    cap = max(cap, prew[c], W - prew[c])
    return seq[:c], seq[c:], cap


def _refine_units(U: _Units, seq, V1, V2, cap):
    """Single-unit moves with positive gain in L(V1) + L(V2): V1 stays a
    down-set of the sequence's units, both sides non-empty and within the
    weight cap; ties by the unit's smaller min gate; at most 4|seq| moves."""
    dag = U.dag
    inP = set(seq)
    side = {}
    for u in V1:
        side[u] = 1
    for u in V2:
        side[u] = 2
    n = dag.n
    cnt = {1: [0] * n, 2: [0] * n}
    use = {}
    for u in seq:
        uq = {}
        for g in U.gates[u]:
            for q in dag.qubits[g]:
                uq[q] = uq.get(q, 0) + 1
        use[u] = uq
        for q, c in uq.items():
            cnt[side[u]][q] += c
    size = {1: len(V1), 2: len(V2)}
    wt = {1: sum(len(U.gates[u]) for u in V1), 2: sum(len(U.gates[u]) for u in V2)}
    order = sorted(seq, key=lambda u: U.mg[u])
    moves = 0
    limit = 4 * len(seq)
    while moves < limit:
        best = None
        for u in order:
            s = side[u]
            o = 3 - s
            if size[s] == 1 or wt[o] + len(U.gates[u]) > cap:
                continue
            if s == 1:
                if any(x in inP and side[x] == 1 for x in U.succ[u]):
                    continue
            else:
                if any(x in inP and side[x] == 2 for x in U.pred[u]):
                    continue
            gain = 0
            for q, c in use[u].items():
                if cnt[s][q] == c:
                    gain += 1
                if cnt[o][q] == 0:
                    gain -= 1
            if gain > 0 and (best is None or gain > best[0]):
                best = (gain, u)
        if best is None:
            break
        u = best[1]
        s = side[u]
        o = 3 - s
        for q, c in use[u].items():
            cnt[s][q] -= c
            cnt[o][q] += c
        side[u] = o
        size[s] -= 1
        size[o] += 1
        wt[s] -= len(U.gates[u])
        wt[o] += len(U.gates[u])
        moves += 1
    A = [u for u in seq if side[u] == 1]
    B = [u for u in seq if side[u] == 2]
    return A, B


def _rb_units(U: _Units, seq, k, leaves):
    """Recursive bisection of a unit sequence until L <= k; leaves are
    emitted V1 subtree first, then V2."""
    stack = [seq]
    while stack:
        seq = stack.pop()
        m = 0
        for u in seq:
            m |= U.qm[u]
        if bin(m).count("1") <= k:
            leaves.append([g for u in seq for g in U.gates[u]])
            continue
        V1, V2, cap = _bisect_units(U, seq, k)
        V1, V2 = _refine_units(U, seq, V1, V2, cap)
        stack.append(V2)
        stack.append(V1)


def dagp_phases(gates, n, k):
    """The three dagP phases; returns (clusters, rb_leaves, merged_parts),
    each a list of gate lists.

    1. acyclic agglomerative clustering from single gates, merging only
       pairs that share a qubit (coarsening);
    2. recursive bisection of the cluster sequence (Kahn order keyed by the
       smallest gate) until each piece has L <= k;
    3. merge phase over the pieces with all pairs as candidates.
    """
    dag = Dag(gates, n)
    _check_arity(dag, k)
    if dag.G == 0:
        return [], [], []
    U = _Units(dag, [[g] for g in range(dag.G)])
    U.merge_loop(k, zero_shared=False)
    clusters = [U.gates[u] for u in sorted(U.gates, key=lambda u: U.mg[u])]
    seq = _topo_units(U.succ, U.pred, list(U.gates), U.mg)
    leaves = []
    _rb_units(U, seq, k, leaves)
    M = _Units(dag, leaves)
    M.merge_loop(k, zero_shared=True)
    merged = [M.gates[u] for u in sorted(M.gates, key=lambda u: M.mg[u])]
    return clusters, leaves, merged


def dagp(gates, n, k):
    dag = Dag(gates, n)
    _check_arity(dag, k)
    if dag.G == 0:
        return []
    _, _, merged = dagp_phases(gates, n, k)
    return schedule(dag, _parts_to_pog(dag.G, merged))


# ------------------------------------------------------------ schedule ----

def _part_graph(dag: Dag, pog, P):
    succ = [set() for _ in range(P)]
    for g in range(dag.G):
        a = pog[g]
        for s in dag.succs[g]:
            b = pog[s]
            if b != a:
                succ[a].add(b)
    return succ


def schedule(dag: Dag, pog):
    """Renumber parts in Kahn order of the part graph, min-heap keyed by the
    smallest gate index of each part. Returns part_of_gate (list of ints)."""
    if dag.G == 0:
        return []
    P = max(pog) + 1
    mg = [None] * P
    for g in range(dag.G):
        if mg[pog[g]] is None:
            mg[pog[g]] = g
    succ = _part_graph(dag, pog, P)
    indeg = [0] * P
    for a in range(P):
        for b in succ[a]:
            indeg[b] += 1
    h = [(mg[a], a) for a in range(P) if indeg[a] == 0]
    heapq.heapify(h)
    newid = [-1] * P
    nxt = 0
    while h:
        _, a = heapq.heappop(h)
        newid[a] = nxt
        nxt += 1
        for b in succ[a]:
            indeg[b] -= 1
            if indeg[b] == 0:
                heapq.heappush(h, (mg[b], b))
    if nxt != P:
        raise PartitionError("part graph has a cycle")
    return [newid[p] for p in pog]


def beam(gates, n, k, width=16):
    """The repository's beam-search builder, written from its definition (it
    is an addition, not one of the paper's three builders). A partition is a
    chain of down-sets D_0 = {} < D_1 < ... < D_P = all gates; a step adds
    one part X = D_{i+1} - D_i.

    closure(D, Q): every gate whose qubits lie in Q and whose predecessors
    are in D or the closure (the largest such set).
    From a kept prefix D, every available gate g0 (ascending) seeds one
    candidate: Q = qubits(g0), then while |Q| < k, among the qubits (not in
    Q) of the gates outside closure(D, Q) whose predecessors are all in it,
    add the one whose closure adds the most gates (the smallest such qubit);
    at width >= 32, while two more qubits fit, a qubit q scores
    1024 * (most gates added by closure(D, Q + q + q2) over the same kind of
    follow-up qubit q2, or by closure(D, Q + q) if larger) + gates added by
    closure(D, Q + q). The candidate is D + closure(D, Q) if that adds a gate;
    a down-set reached twice keeps its first parent (kept prefixes in order,
    seeds ascending). Each level keeps the `width` candidates covering the
    most gates, ties to the smaller gate set compared as 64-gate words from
    gate 0 (bit 63 of a word most significant); the first kept candidate
    covering every gate ends the search. Parts are then numbered by
    ``schedule``."""
    dag = Dag(gates, n)
    _check_arity(dag, k)
    G = dag.G
    if G == 0:
        return []
    if width < 1:
        width = 16
    W = (G + 63) // 64
    full = (1 << G) - 1

    def closure(D, Q):
        E = D
        for g in range(G):   # gate order is topological: one sweep reaches the fixed point
            if (E >> g) & 1 or dag.qmask[g] & ~Q:
                continue
            if all((E >> p) & 1 for p in dag.preds[g]):
                E |= 1 << g
        return E

    def blocked_qubits(E):
        m = 0
        for h in range(G):
            if not (E >> h) & 1 and all((E >> p) & 1 for p in dag.preds[h]):
                m |= dag.qmask[h]
        return m

    def popcount(x):
        return bin(x).count("1")

    def words(E):
        return tuple((E >> (64 * i)) & ((1 << 64) - 1) for i in range(W))

    nodes = [(0, None)]       # (down-set, parent node): a down-set can recur at a later level
    level = [(0, 0, 0)]       # (down-set, gates covered, node)
    while True:
        cand = {}             # down-set -> (gates covered, parent node); first insertion kept
        order = []
        for D, cnt, node in level:
            avail = [g for g in range(G) if not (D >> g) & 1 and all((D >> p) & 1 for p in dag.preds[g])]
            for g0 in avail:
                Q = dag.qmask[g0]
                E = closure(D, Q)
                while popcount(Q) < k:
                    cq = blocked_qubits(E) & ~Q
                    if not cq:
                        break
                    look = width >= 32 and popcount(Q) + 2 <= k
                    best_q, best_s = -1, -1
                    for q in range(n):
                        if not (cq >> q) & 1:
                            continue
                        E1 = closure(D, Q | (1 << q))
                        added = popcount(E1) - popcount(D)
                        score = added
                        if look:
                            best2 = added
                            cq2 = blocked_qubits(E1) & ~(Q | (1 << q))
                            for q2 in range(n):
                                if (cq2 >> q2) & 1:
                                    E2 = closure(D, Q | (1 << q) | (1 << q2))
                                    best2 = max(best2, popcount(E2) - popcount(D))
                            score = best2 * 1024 + added
                        if score > best_s:
                            best_q, best_s = q, score
                    Q |= 1 << best_q
                    E = closure(D, Q)
                if E == D or E in cand:
                    continue
                cand[E] = (popcount(E), node)
                order.append(E)
        order.sort(key=lambda E: (-cand[E][0], words(E)))
        level = []
        for E in order[:width]:
            nodes.append((E, cand[E][1]))
            level.append((E, cand[E][0], len(nodes) - 1))
        done = [node for E, c, node in level if c == G]
        if done:
            break
    chain = []
    node = done[0]
    while node:
        chain.append(nodes[node][0])
        node = nodes[node][1]
    chain.reverse()
    pog = [0] * G
    prev = 0
    for i, E in enumerate(chain):
        X = E & ~prev
        for g in range(G):
            if (X >> g) & 1:
                pog[g] = i
        prev = E
    return schedule(dag, pog)


def partition(gates, n, method, k, seed=0, trials=16):
    if method == "nat":
        return nat(gates, n, k)
    if method == "dfs":
        return dfs(gates, n, k, seed=seed, trials=trials)
    if method == "dagp":
        return dagp(gates, n, k)
    if method == "beam":
        return beam(gates, n, k, width=trials)
    raise ValueError(method)


def multilevel(gates, n, m1, k1, m2, k2, seed=0, trials=16):
    """Multi-level partitioning (Sec. IV-B): the circuit is partitioned with
    builder m1 under the first-level limit k1; then each first-level part,
    taken as a circuit of its own (its gates in their original order), is
    partitioned again with builder m2 under the second-level limit k2.
    Returns (outer, inner): the first-level part of every gate, and its
    second-level part numbered over the whole circuit (first-level parts in
    schedule order, then each part's own schedule)."""
    outer = partition(gates, n, m1, k1, seed=seed, trials=trials)
    P = (max(outer) + 1) if len(outer) else 0
    inner = [0] * len(gates)
    base = 0
    for p in range(P):
        ids = [g for g in range(len(gates)) if outer[g] == p]
        sub = [gates[g] for g in ids]
        sp = partition(sub, n, m2, k2, seed=seed, trials=trials)
        for g, x in zip(ids, sp):
            inner[g] = base + x
        base += max(sp) + 1
    return list(outer), inner


# ---------------------------------------------------------- validation ----

def check_partition(gates, n, k, pog):
    """Validity conditions of the acyclic partitioning problem (Sec. IV-A)
    plus the schedule property. Returns the number of parts; raises
    AssertionError on a violation."""
    dag = Dag(gates, n)
    G = dag.G
    assert len(pog) == G
    if G == 0:
        return 0
    P = max(pog) + 1
    members = [[] for _ in range(P)]
    for g, p in enumerate(pog):
        assert 0 <= p < P
        members[p].append(g)
    for p in range(P):
        assert members[p], f"part {p} empty"
        L = working_set(dag, members[p])
        assert L <= k, f"part {p}: L={L} > k={k}"
        assert working_set_by_edges(dag, members[p]) == L, f"part {p}: edge count != L"
    for g in range(G):
        for s in dag.succs[g]:
            assert pog[s] >= pog[g], f"edge {g}->{s} goes from part {pog[g]} back to {pog[s]}"
    return P


def brute_force_min_parts(gates, n, k):
    """Minimum number of parts of an acyclic partition with L <= k, by BFS
    over down-sets: parts listed in a topological order of the part graph
    have down-set prefixes, so a partition is a chain of down-sets.
    Exponential; for DAGs of at most ~16 gates."""
    dag = Dag(gates, n)
    _check_arity(dag, k)
    G = dag.G
    full = (1 << G) - 1
    predmask = [0] * G
    for g in range(G):
        for p in dag.preds[g]:
            predmask[g] |= 1 << p
    dist = {0: 0}
    frontier = [0]
    while frontier:
        nxt = []
        for D in frontier:
            d = dist[D]
            # enumerate non-empty X (added in increasing id) with D|X a down-set, L(X) <= k
            def ext(X, qmask, start):
                for g in range(start, G):
                    bit = 1 << g
                    if (D | X) & bit:
                        continue
                    if predmask[g] & ~(D | X):
                        continue
                    m = qmask | dag.qmask[g]
                    if bin(m).count("1") > k:
                        continue
                    Y = X | bit
                    E = D | Y
                    if E not in dist:
                        dist[E] = d + 1
                        nxt.append(E)
                    ext(Y, m, g + 1)
            ext(0, 0, 0)
        if full in dist:
            return dist[full]
        frontier = nxt
    return dist.get(full, 0)
