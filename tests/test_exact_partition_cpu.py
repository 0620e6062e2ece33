"""The exact part builder (SV_PART_EXACT, the optimum of Sec. V-A's ILP
comparison) against the oracle's independent brute force over down-sets,
the validity conditions of an acyclic partition, and the heuristics (Nat,
DFS, dagP) it must never beat. CPU only: the host library partitions."""
import random

import pytest

import synth
from oracle import partition as pt
from paper_2205_06973_gb300 import _native as N
from paper_2205_06973_gb300 import api


def _rand(n, G, seed):
    r = random.Random(seed)
    g = []
    for _ in range(G):
        if r.random() < 0.5:
            a, b = r.sample(range(n), 2)
            g.append(("CX", (a, b), 0.0))
        else:
            g.append((r.choice(("H", "RZ")), (r.randrange(n),), 0.3))
    return g


def _parts(g, n, method, k):
    p = api.Plan(g, n, method, k)
    pog, P = p.export()
    p.close()
    return [int(x) for x in pog], P


def test_exact_equals_brute_force_and_is_valid():
    for seed in range(40):
        n = 5 + seed % 3
        G = 9 + seed % 7
        k = 2 + seed % 3
        g = _rand(n, G, 100 + seed)
        pog, P = _parts(g, n, "exact", k)
        assert P == pt.brute_force_min_parts(g, n, k), seed
        assert pt.check_partition(g, n, k, pog) == P


def test_heuristics_never_beat_the_optimum():
    cases = [(8, synth.qft(8), 4), (8, synth.layered(8, 4, seed=3), 4), (8, synth.param(8, 3, seed=2), 4),
             (6, synth.qft(6), 3)]
    for n, g, k in cases:
        _, opt = _parts(g, n, "exact", k)
        for m in ("nat", "dfs", "dagp"):
            assert _parts(g, n, m, k)[1] >= opt, (n, k, m)


def test_exact_special_cases():
    # one part when k covers every qubit; one gate per part when no two fit
    g = _rand(6, 20, 7)
    assert _parts(g, 6, "exact", 6)[1] == 1
    chain = [("CX", (i, i + 1), 0.0) for i in range(5)]
    assert _parts(chain, 6, "exact", 2)[1] == 5
    # a CX ladder behind an H: parts of three qubits hold two rungs each
    ghz = [("H", (0,), 0.0)] + chain
    assert _parts(ghz, 6, "exact", 3)[1] == 3 == pt.brute_force_min_parts(ghz, 6, 3)


def test_exact_refuses_large_circuits():
    g = _rand(8, 300, 1)
    with pytest.raises(N.SvError) as e:
        api.Plan(g, 8, "exact", 4)
    assert e.value.status == N.SV_ERR_ARG


def test_beam_builder_valid_deterministic_and_near_optimal():
    """The beam builder (SV_PART_BEAM) gives valid acyclic partitions, the
    same one on every call, never fewer parts than the optimum, and on the
    small family instances at most one part more."""
    cases = [(8, synth.qft(8), 4), (10, synth.layered(10, 6, seed=5), 5), (10, synth.param(10, 4, seed=4), 5),
             (10, synth.qft(10), 4)]
    for n, g, k in cases:
        _, opt = _parts(g, n, "exact", k)
        pog, P = _parts(g, n, "beam", k)
        assert pt.check_partition(g, n, k, pog) == P
        assert _parts(g, n, "beam", k) == (pog, P)
        assert opt <= P <= opt + 1, (n, k, P, opt)
    for seed in range(20):
        n, k = 6, 3
        g = _rand(n, 14, 300 + seed)
        pog, P = _parts(g, n, "beam", k)
        assert pt.check_partition(g, n, k, pog) == P >= pt.brute_force_min_parts(g, n, k)


def test_beam_builder_on_the_benchmark_circuits():
    """Fewer parts than dagP on the 28-qubit layered circuit and the 33-qubit
    QFT (the passes of the benchmark steps), and a valid partition."""
    n, g = synth.layered_28q()
    p = api.Plan(g, n, "beam", 6, dfs_trials=64)
    pog, P = p.export()
    p.close()
    assert pt.check_partition(g, n, 6, [int(x) for x in pog]) == P
    assert P < _parts(g, n, "dagp", 6)[1]
    q = synth.qft(33)
    assert _parts(q, 33, "beam", 6)[1] < _parts(q, 33, "dagp", 6)[1]


def test_beam_builder_bit_exact_with_oracle():
    """The C++ beam builder against the oracle's own implementation of the
    same definition: the same part of every gate, for widths 1, 4, 16 and
    32 (the look-ahead), on the three families and on a 252-gate circuit
    whose gate sets span four 64-bit words."""
    cases = [(8, synth.qft(8), 4), (8, synth.layered(8, 4, seed=3), 4), (8, synth.param(8, 3, seed=2), 4),
             (10, synth.qft(10), 5), (10, synth.layered(10, 5, seed=5), 5), (10, synth.param(10, 4, seed=4), 5)]
    for n, g, k in cases:
        for w in (1, 4, 16, 32):
            p = api.Plan(g, n, "beam", k, dfs_trials=w)
            pog = [int(x) for x in p.export()[0]]
            p.close()
            assert pog == pt.beam(g, n, k, w), (n, k, w)
    n, g = 12, synth.layered(12, 14, seed=9)
    for w in (4, 32):
        p = api.Plan(g, n, "beam", 6, dfs_trials=w)
        pog = [int(x) for x in p.export()[0]]
        p.close()
        assert pog == pt.beam(g, n, 6, w), w
