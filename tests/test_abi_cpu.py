"""C-ABI checks that need no GPU: the library loads, exports every entry
point declared in include/hisvsim.h, the host partitioners agree bit-exactly
with the oracle's, and argument errors come back as status codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle import partition as pt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2205_06973_gb300 import build
    build.build()
    from paper_2205_06973_gb300 import _native
    return _native


def header_symbols():
    syms = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            syms |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(sv_\w+)\s*\(", txt, flags=re.M))
    return sorted(syms)


def test_exports_every_declared_symbol(native):
    syms = header_symbols()
    assert "sv_create" in syms and "sv_apply_parts" in syms and "sv_measure_probs" in syms
    for s in syms:
        assert hasattr(native.lib, s), s


def test_version(native):
    assert b"sm_103a" in native.lib.sv_version()


def _plan(native, gates, n, method, k, seed=0, trials=16):
    from paper_2205_06973_gb300.api import Plan
    return Plan(gates, n, method, k, seed=seed, dfs_trials=trials)


def _rand(n, G, seed):
    r = synth.SplitMix64(seed)
    out = []
    for _ in range(G):
        c = r.randint(4)
        if c == 0:
            out.append((("H", "RX", "RZ", "T")[r.randint(4)], (r.randint(n),), r.angle()))
        else:
            a = r.randint(n)
            b = (a + 1 + r.randint(n - 1)) % n
            out.append((("CX", "CZ", "CP", "SWAP")[r.randint(4)], (a, b), r.angle()))
    return out


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("method", ["nat", "dfs", "dagp"])
def test_partition_bit_exact_random(native, seed, method):
    n = 9 + seed % 5
    k = 2 + seed % 6
    g = _rand(n, 200 + 30 * seed, 500 + seed)
    p = _plan(native, g, n, method, k, seed=seed, trials=4 + seed)
    pog, P = p.export()
    ref = pt.partition(g, n, method, k, seed=seed, trials=4 + seed)
    assert list(pog) == ref
    assert P == max(ref) + 1
    pt.check_partition(g, n, k, ref)


@pytest.mark.parametrize("k", [8, 10, 12])
@pytest.mark.parametrize("method", ["nat", "dfs", "dagp"])
def test_partition_bit_exact_layered_28(native, method, k):
    n, g = synth.layered_28q()
    pog, P = _plan(native, g, n, method, k).export()
    assert list(pog) == pt.partition(g, n, method, k, seed=0)


@pytest.mark.parametrize("k", [6, 12])
def test_partition_bit_exact_qft_33(native, k):
    n, g, _ = synth.qft_basis(33)
    for method in ("nat", "dfs", "dagp"):
        pog, P = _plan(native, g, n, method, k).export()
        assert list(pog) == pt.partition(g, n, method, k, seed=0)


def test_partition_bit_exact_param_batch(native):
    for i in range(6):
        n, g = synth.batch_circuit(i)
        for method in ("nat", "dagp"):
            pog, _ = _plan(native, g, n, method, 10).export()
            assert list(pog) == pt.partition(g, n, method, 10)


def test_plan_errors(native):
    from paper_2205_06973_gb300.api import Plan
    with pytest.raises(native.SvError) as e:
        Plan([("CX", (0, 1), 0.0)], 2, "dagp", 1)
    assert e.value.status == native.SV_ERR_PARTITION
    with pytest.raises(native.SvError) as e:
        Plan([("H", (3,), 0.0)], 2, "nat", 2)
    assert e.value.status == native.SV_ERR_ARG
    with pytest.raises(native.SvError) as e:
        Plan([("CX", (1, 1), 0.0)], 2, "nat", 2)
    assert e.value.status == native.SV_ERR_ARG
    arr = native.encode_gates([("CX", (0, 1), 0.0)])
    arr[0].arity = 1
    h = ctypes.c_void_p()
    st = native.lib.sv_plan_build(ctypes.cast(arr, ctypes.c_void_p), 1, 2, native.SV_PART_NAT, 2, 0, 0,
                                  ctypes.byref(h))
    assert st == native.SV_ERR_ARG
    assert b"arity" in native.lib.sv_last_error()


def test_plan_stats_counts(native):
    n, g = synth.layered_28q(n=16, depth=10)
    p = _plan(native, g, n, "dagp", 8)
    s = p.stats("c64", 12)
    pog, P = p.export()
    assert s["passes"] == P and s["dense"] == 0
    d = p.stats("c64", 12, tc=True)
    assert d["passes"] == P and 0 < d["dense"] <= P
    assert s["phases"] >= P
    # every op comes from at least one gate (runs of one-qubit gates and of
    # diagonal gates merge), plus at most one per-thread-phase op per phase
    assert 0 < s["ops"] <= len(g) + s["phases"]


def test_plan_tile_too_small(native):
    n, g = synth.layered_28q(n=20, depth=4)
    p = _plan(native, g, n, "dagp", 12)
    with pytest.raises(native.SvError):
        p.stats("c128", 11)    # a 12-qubit part cannot fit an 11-qubit tile


@pytest.mark.parametrize("k", [4, 6, 10])
def test_partition_bit_exact_serving_requests(native, k):
    """Large requests of the serving stream (parameterised, layered and QFT
    families, 21-22 qubits, ~1500 gates) at the part sizes the server uses."""
    seen = set()
    i = 0
    while len(seen) < 3 and i < 400:
        n, fam, g = synth.serving_request(i, seed=5)
        i += 1
        if n > 22 or n < 21 or fam in seen:
            continue
        seen.add(fam)
        pog, _ = _plan(native, g, n, "dagp", k).export()
        ref = pt.partition(g, n, "dagp", k)
        assert list(pog) == ref, (i - 1, fam)
        pt.check_partition(g, n, k, ref)


def test_plan_stats_from_many_threads(native):
    """The plan's program caches fill on first use; concurrent callers of one
    plan get the same answer."""
    import concurrent.futures as cf
    n, g = synth.layered_28q(n=16, depth=10)
    p = _plan(native, g, n, "dagp", 8)
    with cf.ThreadPoolExecutor(8) as ex:
        res = list(ex.map(lambda i: p.stats("c64" if i % 2 else "c128", 12, tc=bool(i % 3 == 0)), range(64)))
    ref = {(i % 2, i % 3 == 0): r for i, r in enumerate(res)}
    for i, r in enumerate(res):
        assert r == ref[(i % 2, i % 3 == 0)]


def test_cost_model_picks_kernel_per_circuit(native):
    """The serving cost model (host only) keeps the candidate it estimates
    fastest: a ring of CZ gates (diagonal, one op each on the gate-list
    kernel, k = 10 covers more of the ring per pass) goes to the gate-list
    plan; a random layered circuit and, with beam-search plans, the QFT (60
    dense passes at 33 qubits: 1.29 s against 1.46 s on the gate-list kernel,
    measured) to the tensor-core plan."""
    from paper_2205_06973_gb300 import autotune
    n = 24
    ring = [("CZ", (q, (q + 1) % n), 0.0) for q in range(n)] * 3
    plan, tc, est, jit = autotune.choose_plan(ring, n)
    assert not tc and not jit and len(est) == 2 and est[1]["est_s"] < est[0]["est_s"]
    plan.close()
    for n, g in (synth.layered_28q(n=24, depth=30), synth.qft_basis(26)[:2]):
        plan, tc, est, jit = autotune.choose_plan(g, n)
        assert tc and not jit and est[0]["est_s"] < est[1]["est_s"]
        plan.close()
    # specialised candidates only from 29 qubits on (their compilation is
    # host time that a smaller state's passes do not repay); choose_plan
    # estimates them without compiling
    plan, tc, est, jit = autotune.choose_plan(synth.qft_basis(30)[1], 30)
    assert len(est) == 4 and any(e["jit"] for e in est)
    plan.close()


def test_new_builders_and_batch_entry_points_validate_arguments(native):
    """Argument checks that need no device: an unknown method, the exact and
    beam builders on an empty circuit and with k below a gate's arity, the
    beam width default, and the dense batch entry points on a NULL batch."""
    from paper_2205_06973_gb300.api import Plan
    arr = native.encode_gates([("H", (0,), 0.0)])
    h = ctypes.c_void_p()
    st = native.lib.sv_plan_build(ctypes.cast(arr, ctypes.c_void_p), 1, 2, 6, 2, 0, 0, ctypes.byref(h))
    assert st == native.SV_ERR_ARG and b"method" in native.lib.sv_last_error()
    for m in ("exact", "beam"):
        p = Plan([], 3, m, 2)
        assert p.export()[1] == 0
        p.close()
        with pytest.raises(native.SvError) as e:
            Plan([("CX", (0, 1), 0.0)], 2, m, 1)
        assert e.value.status == native.SV_ERR_PARTITION
    g = [("H", (q,), 0.0) for q in range(4)] + [("CX", (q, q + 1), 0.0) for q in range(3)]
    a = Plan(g, 4, "beam", 2, dfs_trials=0).export()
    b = Plan(g, 4, "beam", 2, dfs_trials=16).export()
    assert list(a[0]) == list(b[0]) and a[1] == b[1]
    assert native.lib.sv_batch_set_dense(None, 13, 0, 0) == native.SV_ERR_ARG
    n1, n2, n3 = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    assert native.lib.sv_batch_dense_info(None, ctypes.byref(n1), ctypes.byref(n2), ctypes.byref(n3)) == \
        native.SV_ERR_ARG


@pytest.mark.parametrize("m1,k1,m2,k2", [("nat", 8, "nat", 4), ("dagp", 10, "dagp", 5), ("dfs", 8, "dagp", 4),
                                         ("dagp", 12, "beam", 5), ("beam", 10, "dfs", 5)])
def test_multilevel_bit_exact(native, m1, k1, m2, k2):
    """sv_plan_build_ml gives the oracle's two-level partition gate for gate
    (both levels), on a random circuit and on the 28-qubit layered one."""
    from paper_2205_06973_gb300.api import Plan
    cases = [(12, _rand(12, 400, 77))]
    if "beam" not in (m1, m2):     # the oracle's beam builder is slow at 2520 gates
        cases.append(synth.layered_28q())
    for n, g in cases:
        p = Plan(g, n, m1, k1, inner=(m2, k2))
        outer, P = p.export()
        inner, Q = p.export_inner()
        ro, ri = pt.multilevel(g, n, m1, k1, m2, k2)
        assert list(outer) == ro and list(inner) == ri
        assert P == max(ro) + 1 and Q == max(ri) + 1
        pt.check_partition(g, n, k2, list(inner))
        p.close()


def test_multilevel_errors(native):
    from paper_2205_06973_gb300.api import Plan
    g = [("CX", (0, 1), 0.0), ("H", (2,), 0.0)]
    with pytest.raises(native.SvError) as e:
        Plan(g, 3, "dagp", 3, inner=("dagp", 4))      # k2 > k1
    assert e.value.status == native.SV_ERR_ARG
    with pytest.raises(native.SvError) as e:
        Plan(g, 3, "dagp", 3, inner=("dagp", 1))      # a two-qubit gate under k2 = 1
    assert e.value.status == native.SV_ERR_PARTITION
    with pytest.raises(native.SvError) as e:
        Plan(g, 3, "dagp", 3).export_inner()          # one-level plan
    assert e.value.status == native.SV_ERR_ARG
    p = Plan(synth.layered(14, 4, seed=2), 14, "dagp", 10, inner=("dagp", 6))
    with pytest.raises(native.SvError) as e:          # second-level parts wider than the register bits
        p.stats("c64")
    assert e.value.status == native.SV_ERR_PARTITION
    p.close()


@pytest.mark.parametrize("precision,k,expect", [("c64", 8, 12), ("c64", 10, 12), ("c64", 11, 13), ("c64", 12, 13),
                                                ("c128", 8, 11), ("c128", 10, 11), ("c128", 11, 12),
                                                ("c128df", 12, 12)])
def test_default_tile_fills_sectors(native, precision, k, expect):
    """Default tile: the largest part plus the lowest free qubits that make a
    contiguous run of the tile fill a 32-byte sector (two for complex64, one
    for the 16-byte forms), at least 2^12 / 2^11 and at most 2^13 / 2^12.
    The generated source of a part names its tile size, so the default's
    source equals the source for the expected tile and no other."""
    n, g = synth.layered_28q(n=18, depth=8)
    p = _plan(native, g, n, "dfs", k)
    assert p.stats(precision)["passes"] > 0
    src = p.source(0, precision)
    assert src == p.source(0, precision, expect)
    tmax = 13 if precision == "c64" else 12
    for t in range(max(k, 10), tmax + 1):
        if t != expect:
            assert src != p.source(0, precision, t)
    p.close()


def test_random_gate_arrays_return_a_status(native):
    """Random, mostly invalid, gate arrays (unknown kinds, arities 0-4,
    qubits past n, non-finite angles, n and k out of range, unknown
    builders) through sv_plan_build / sv_plan_build_ml and, where a plan
    results, its export, statistics and generated source: every call returns
    a status and none crashes. (Also run clean at 4000 arrays per seed under
    AddressSanitizer and UndefinedBehaviorSanitizer builds of the host
    code.)"""
    import math
    import random
    L = native.lib
    r = random.Random(11)
    nk = len(native.KIND)
    seen = set()
    for _ in range(300):
        n = r.choice([0, 1, 2, 3, 5, 8, 12, 14, 36, 37, -1])
        G = r.choice([0, 1, 2, 5, 20, 60])
        arr = (native.sv_gate * max(1, G))()
        for i in range(G):
            g = arr[i]
            g.kind = r.randint(0, nk + 2) if r.random() < 0.1 else r.randint(0, nk - 1)
            g.arity = r.choice([0, 1, 2, 3, 4]) if r.random() < 0.1 else r.choice([1, 2])
            for j in range(3):
                g.q[j] = r.randint(0, max(0, n + 1)) if r.random() < 0.1 else r.randint(0, max(0, n - 1))
            g.theta = r.choice([0.0, math.pi, float("nan"), float("inf"), r.uniform(-10, 10)])
        method, k = r.randint(-1, 6), r.choice([0, 1, 2, 3, 5, 6, 9, 12, 40])
        h = ctypes.c_void_p()
        st = L.sv_plan_build(ctypes.cast(arr, ctypes.c_void_p), G, n, method, k, 0, r.choice([0, 4]), ctypes.byref(h))
        h2 = ctypes.c_void_p()
        st2 = L.sv_plan_build_ml(ctypes.cast(arr, ctypes.c_void_p), G, n, method, k, r.randint(-1, 6),
                                 r.choice([0, 1, 3, 5]), 0, 4, ctypes.byref(h2))
        seen |= {st, st2}
        for hh, ok in ((h, st == native.SV_OK), (h2, st2 == native.SV_OK)):
            if not ok:
                assert not hh.value
                continue
            pog = (ctypes.c_uint32 * max(1, G))()
            P = ctypes.c_uint32()
            assert L.sv_plan_export(hh, pog, G, ctypes.byref(P)) == native.SV_OK
            assert all(pog[i] < P.value for i in range(G))
            a, b, c, d = (ctypes.c_uint32() for _ in range(4))
            for prec in (0, 1, 2):
                L.sv_plan_stats(hh, prec, 0, 0, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d))
            if n >= 10:
                buf = ctypes.create_string_buffer(1 << 16)
                ln = ctypes.c_size_t()
                L.sv_plan_source(hh, 0, 0, 0, 0, buf, 1 << 16, ctypes.byref(ln))
            assert L.sv_plan_destroy(hh) == native.SV_OK
    assert native.SV_OK in seen and native.SV_ERR_ARG in seen
