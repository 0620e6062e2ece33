"""Pins of the oracle's part builders (Sec. IV) against hand-derived examples,
the validity conditions of the acyclic partitioning problem and a brute-force
minimum on tiny DAGs."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import partition as pt
from oracle import partition as P
from oracle import sim

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "partition_examples.json")


def _load():
    with open(GOLDEN) as f:
        ex = json.load(f)["examples"]
    for e in ex:
        e["gates"] = [(g[0], tuple(g[1]), g[2]) for g in e["gates"]]
    return ex


@pytest.mark.parametrize("ex", _load(), ids=lambda e: e["name"])
def test_hand_examples(ex):
    n, k, g = ex["n"], ex["k"], ex["gates"]
    assert pt.nat(g, n, k) == ex["nat_part_of_gate"]
    assert pt.brute_force_min_parts(g, n, k) == ex["optimum_parts"]
    for m in ("nat", "dfs", "dagp"):
        pog = pt.partition(g, n, m, k, seed=1)
        P = pt.check_partition(g, n, k, pog)
        assert P >= ex["optimum_parts"]
    assert max(pt.dagp(g, n, k)) + 1 == ex["optimum_parts"]


def test_working_set_example_of_sec4():
    """Gate A on (q0, q1) and gate B on (q0, q2) need 3 qubits together."""
    g = [("CX", (0, 1), 0.0), ("CZ", (0, 2), 0.0)]
    dag = pt.Dag(g, 3)
    assert pt.working_set(dag, [0, 1]) == 3
    assert pt.working_set_by_edges(dag, [0, 1]) == 3
    assert pt.working_set_by_edges(dag, [1]) == 2   # in-edge on q0 + entry of q2


def _rand(n, G, seed):
    r = synth.SplitMix64(seed)
    out = []
    for _ in range(G):
        if r.randint(3) == 0:
            out.append(("H", (r.randint(n),), 0.0))
        else:
            a = r.randint(n)
            b = (a + 1 + r.randint(n - 1)) % n
            out.append((("CX", "CZ")[r.randint(2)], (a, b), 0.0))
    return out


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("k", [2, 3, 4, 6])
def test_validity_random(seed, k):
    n = 8
    g = _rand(n, 150, 1000 + seed)
    for m in ("nat", "dfs", "dagp"):
        pog = pt.partition(g, n, m, k, seed=seed)
        pt.check_partition(g, n, k, pog)


def test_validity_workloads():
    n, g = synth.layered_28q(n=16, depth=12)
    for k in (4, 8):
        for m in ("nat", "dfs", "dagp"):
            pt.check_partition(g, n, k, pt.partition(g, n, m, k, seed=3))
    n, g = 14, synth.qft(14)
    for m in ("nat", "dfs", "dagp"):
        pt.check_partition(g, n, 6, pt.partition(g, n, m, 6, seed=3))


def test_brute_force_against_heuristics():
    """Every builder is >= the optimum; dagP reaches it on most tiny DAGs
    (the paper reports the optimum on 48 of 52 ILP cases)."""
    hits = total = 0
    for seed in range(40):
        n = 5
        g = _rand(n, 11, 50 + seed)
        k = 2 + seed % 3
        opt = pt.brute_force_min_parts(g, n, k)
        for m in ("nat", "dfs"):
            assert max(pt.partition(g, n, m, k, seed=seed)) + 1 >= opt
        d = max(pt.dagp(g, n, k)) + 1
        assert d >= opt
        hits += d == opt
        total += 1
    assert hits >= 0.75 * total, (hits, total)


def test_brute_force_small_cases():
    # one gate per part when no two gates fit together
    g = [("CX", (0, 1), 0.0), ("CX", (1, 2), 0.0), ("CX", (2, 3), 0.0)]
    assert pt.brute_force_min_parts(g, 4, 2) == 3
    assert pt.brute_force_min_parts(g, 4, 4) == 1
    assert pt.brute_force_min_parts(g, 4, 3) == 2


def test_arity_error():
    g = [("CX", (0, 1), 0.0)]
    for m in ("nat", "dfs", "dagp"):
        with pytest.raises(pt.PartitionError):
            pt.partition(g, 2, m, 1)
    with pytest.raises(pt.PartitionError):
        pt.Dag([("CX", (0, 0), 0.0)], 2)
    with pytest.raises(pt.PartitionError):
        pt.Dag([("H", (5,), 0.0)], 2)


def test_schedule_is_min_gate_kahn():
    g = _rand(6, 60, 77)
    pog = pt.dagp(g, 6, 3)
    P = max(pog) + 1
    first = [min(i for i, p in enumerate(pog) if p == q) for q in range(P)]
    dag = pt.Dag(g, 6)
    # whenever two parts are both ready, the one with the smaller first gate runs first:
    # replay Kahn and compare
    import heapq
    succ = [set() for _ in range(P)]
    for a in range(dag.G):
        for b in dag.succs[a]:
            if pog[a] != pog[b]:
                succ[pog[a]].add(pog[b])
    indeg = [0] * P
    for a in range(P):
        for b in succ[a]:
            indeg[b] += 1
    h = [(first[a], a) for a in range(P) if indeg[a] == 0]
    heapq.heapify(h)
    order = []
    while h:
        _, a = heapq.heappop(h)
        order.append(a)
        for b in succ[a]:
            indeg[b] -= 1
            if indeg[b] == 0:
                heapq.heappush(h, (first[b], b))
    assert order == list(range(P))


def test_dfs_deterministic_and_trials():
    n, g = synth.layered_28q(n=12, depth=8)
    a = pt.dfs(g, n, 5, seed=11, trials=8)
    b = pt.dfs(g, n, 5, seed=11, trials=8)
    assert a == b
    one = max(pt.dfs(g, n, 5, seed=11, trials=1)) + 1
    many = max(pt.dfs(g, n, 5, seed=11, trials=8)) + 1
    assert many <= one


def test_dagp_quality_on_layered():
    """dagP gives no more parts than Nat on the layered and QFT families."""
    n, g = synth.layered_28q(n=20, depth=20)
    for k in (6, 10):
        d = max(pt.dagp(g, n, k)) + 1
        assert d <= max(pt.nat(g, n, k)) + 1
    g = synth.qft(16)
    assert max(pt.dagp(g, 16, 6)) + 1 <= max(pt.nat(g, 16, 6)) + 1


def test_oracle_beam_valid_and_not_below_optimum():
    """The oracle's beam builder is pinned by the validity conditions of the
    partitioning problem and by the brute-force optimum (never fewer parts;
    it is a heuristic: each prefix grows one greedy candidate per available
    gate, so even an unlimited width need not reach the optimum, and on
    these tiny DAGs it mostly does)."""
    hits = 0
    for seed in range(25):
        n = 5
        g = _rand(n, 10, 700 + seed)
        k = 2 + seed % 3
        opt = pt.brute_force_min_parts(g, n, k)
        for w in (1, 4, 1 << 20):
            pog = pt.beam(g, n, k, w)
            assert pt.check_partition(g, n, k, pog) >= opt
        hits += pt.check_partition(g, n, k, pt.beam(g, n, k, 16)) == opt
    assert hits >= 15, hits


# ------------------------------------------------ multi-level (Sec. IV-B) ---

ML_CASES = [("nat", 8, "nat", 4), ("dagp", 8, "dagp", 4), ("dfs", 7, "dagp", 3), ("dagp", 10, "beam", 5),
            ("beam", 9, "nat", 5)]


@pytest.mark.parametrize("m1,k1,m2,k2", ML_CASES)
def test_multilevel_valid_at_both_levels(m1, k1, m2, k2):
    """Both levels satisfy the conditions of Sec. IV-A: the first level under
    k1; each first-level part's inner partition on its own sub-circuit under
    k2; inner parts nest in first-level parts; and the inner parts in order
    form one valid acyclic partition of the whole circuit under k2."""
    n = 11
    g = synth.layered(n, 5, seed=17, two_q=("CX", "CZ"))
    outer, inner = P.multilevel(g, n, m1, k1, m2, k2)
    assert P.check_partition(g, n, k1, outer) == max(outer) + 1
    assert P.check_partition(g, n, k2, inner) == max(inner) + 1
    for x in set(inner):
        assert len({outer[i] for i in range(len(g)) if inner[i] == x}) == 1
    for p in range(max(outer) + 1):
        ids = [i for i in range(len(g)) if outer[i] == p]
        first = min(inner[i] for i in ids)
        P.check_partition([g[i] for i in ids], n, k2, [inner[i] - first for i in ids])
    # the inner numbering follows the first level: part p's inner ids come
    # after part p-1's
    for i in range(len(g)):
        for j in range(len(g)):
            if outer[i] < outer[j]:
                assert inner[i] < inner[j]


def test_multilevel_with_equal_limits_is_one_level():
    """k2 = k1 with the same builder: every first-level part already fits, so
    its re-partition is the part itself and the two levels coincide."""
    n = 10
    g = synth.layered(n, 6, seed=3, two_q=("CX", "CZ"))
    for m in ("nat", "dfs", "dagp"):
        outer, inner = P.multilevel(g, n, m, 6, m, 6)
        assert inner == outer, m


@pytest.mark.parametrize("m1,k1,m2,k2", ML_CASES)
def test_nested_algorithm1_equals_gate_by_gate(m1, k1, m2, k2):
    """Algorithm 1 with nested parts (gather the first-level part's vector,
    run its second-level parts by Algorithm 1 inside it, scatter) gives the
    gate-by-gate state psi_out = U_G ... U_1 psi_in (Sec. II-B)."""
    n = 10
    g = synth.layered(n, 6, seed=5, two_q=("CX", "CZ")) + synth.qft(n)[:40]
    psi = np.asarray(synth.random_amplitudes(n, 4))
    psi = (psi[:, 0] + 1j * psi[:, 1]) / np.linalg.norm(psi[:, 0] + 1j * psi[:, 1])
    outer, inner = P.multilevel(g, n, m1, k1, m2, k2)
    ref = sim.run(n, g, psi)
    out = sim.run_alg1_nested(n, g, outer, inner, psi)
    assert np.abs(out - ref).max() <= 1e-13


def test_nested_algorithm1_catches_a_misplaced_gate():
    """The nested execution is sensitive to the inner order: moving one gate
    into another second-level part against its dependencies changes the
    state (the check above is not vacuous)."""
    n = 6
    g = [("H", (0,), 0.0), ("CX", (0, 1), 0.0), ("RX", (1,), 0.7), ("CZ", (1, 2), 0.0), ("RY", (2,), 1.1)]
    outer = [0, 0, 0, 0, 0]
    good = [0, 0, 1, 1, 1]
    bad = [1, 0, 1, 1, 1]       # H after the CX that depends on it
    ref = sim.run(n, g)
    assert np.abs(sim.run_alg1_nested(n, g, outer, good) - ref).max() <= 1e-13
    assert np.abs(sim.run_alg1_nested(n, g, outer, bad) - ref).max() > 1e-3


def _part_graph(gates, n, pog):
    """Parts' qubit sets and the part graph: an edge a -> b when a gate of a
    is the previous gate on some qubit of a gate of b (the wire order of
    Sec. IV-A), written here from the gate list alone."""
    P = max(pog) + 1
    qs = [set() for _ in range(P)]
    succ = [set() for _ in range(P)]
    last = [None] * n
    for i, (_, qubits, _) in enumerate(gates):
        for q in qubits:
            qs[pog[i]].add(q)
            if last[q] is not None and pog[last[q]] != pog[i]:
                succ[pog[last[q]]].add(pog[i])
            last[q] = i
    return qs, succ


def _reach(succ):
    """reach[a] = the parts reachable from a by a path of length >= 1."""
    P = len(succ)
    reach = [set() for _ in range(P)]
    for a in range(P):
        stack = list(succ[a])
        while stack:
            v = stack.pop()
            if v not in reach[a]:
                reach[a].add(v)
                stack.extend(succ[v])
    return reach


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("k", [3, 4, 6])
def test_nat_cuts_only_where_the_next_gate_overflows(seed, k):
    """Nat (Sec. IV-B, reading R5): parts are runs of the natural gate order,
    and each part ends only because the next gate would take its working
    set above k."""
    n = 8
    g = _rand(n, 120, 2000 + seed)
    pog = pt.partition(g, n, "nat", k)
    run = [pog[0]]
    for i in range(1, len(g)):
        if pog[i] != pog[i - 1]:
            assert pog[i] not in run, "a part is not one run of the gate order"
            run.append(pog[i])
            qs = {q for j in range(len(g)) if pog[j] == pog[i - 1] for q in g[j][1]}
            assert len(qs | set(g[i][1])) > k, i


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("k", [3, 4, 6])
def test_dagp_merge_phase_leaves_no_mergeable_neighbours(seed, k):
    """dagP's merges (reading R7: the clustering of phase 1 and the merge
    phase 3) run until no valid merge of two parts that share a qubit
    remains: for every such pair, either the merged working set exceeds k
    or a path through a third part joins them (merging would close a
    cycle). Validity alone does not see a builder that stops merging early
    (say at k - 1); this does."""
    n = 8
    g = _rand(n, 150, 3000 + seed)
    pog = pt.partition(g, n, "dagp", k)
    qs, succ = _part_graph(g, n, pog)
    reach = _reach(succ)
    P = len(qs)
    for a in range(P):
        for b in range(a + 1, P):
            if not (qs[a] & qs[b]) or len(qs[a] | qs[b]) > k:
                continue
            via = any(b in reach[c] for c in succ[a]) or any(a in reach[c] for c in succ[b])
            assert via, f"parts {a} and {b} could still merge (k={k})"


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("k", [3, 5])
def test_builders_acyclic_by_an_independent_check(seed, k):
    """Acyclicity and the working-set limit of every builder's partition
    (Sec. IV-A), checked by the part graph built above from the gate list
    alone (not the oracle's own checker): no part reaches itself, every
    part has at most k qubits, and the schedule runs a part only after the
    parts it depends on."""
    n = 8
    g = _rand(n, 120, 4000 + seed)
    for m in ("nat", "dfs", "dagp", "beam"):
        pog = pt.partition(g, n, m, k, seed=seed)
        qs, succ = _part_graph(g, n, pog)
        reach = _reach(succ)
        assert all(a not in reach[a] for a in range(len(qs))), m
        assert all(len(q) <= k for q in qs), m
        # part ids are the schedule: every edge goes from an earlier part to a later one
        assert all(b > a for a in range(len(qs)) for b in succ[a]), m


def _wire_preds(gates, n):
    """For each gate, the gates just before it on its qubits (wire order)."""
    last = [None] * n
    preds = []
    for i, (_, qubits, _) in enumerate(gates):
        preds.append({last[q] for q in qubits if last[q] is not None})
        for q in qubits:
            last[q] = i
    return preds


@pytest.mark.parametrize("seed", range(5))
def test_dfs_order_is_a_depth_first_topological_order(seed):
    """The DFS builder's visiting order (Sec. IV-B, reading R6): every gate
    once, after the gates before it on its qubits, and depth first — when a
    gate makes successors ready, the next gate visited is one of them."""
    n = 8
    g = _rand(n, 120, 5000 + seed)
    preds = _wire_preds(g, n)
    dag = P.Dag(g, n)
    order = P.dfs_order(dag, P._SplitMix64(seed))
    assert sorted(order) == list(range(len(g)))
    pos = {x: i for i, x in enumerate(order)}
    assert all(pos[p] < pos[x] for x in range(len(g)) for p in preds[x])
    done = set()
    for i, x in enumerate(order[:-1]):
        done.add(x)
        ready_now = {s for s in range(len(g)) if s not in done and x in preds[s] and preds[s] <= done}
        if ready_now:
            assert order[i + 1] in ready_now, i


def test_dfs_keeps_the_best_trial():
    """DFS over r trials keeps the order with the fewest parts: more trials
    never give more parts, and one trial equals the Nat cut of its order."""
    n = 8
    g = _rand(n, 150, 6000)
    dag = P.Dag(g, n)
    counts = [max(P.dfs(g, n, 4, seed=7, trials=t)) + 1 for t in (1, 2, 4, 16)]
    assert counts == sorted(counts, reverse=True)
    one = P.cut_order(dag, P.dfs_order(dag, P._SplitMix64(7)), 4)
    assert counts[0] == len(one)
