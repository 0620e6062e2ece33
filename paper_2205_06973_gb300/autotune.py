"""Autotuner: picks the part limit k and the launch shape by measuring them.

* ``tune_state`` times candidate (method, k, tensor-core dense path, tile)
  configurations of one circuit on one state with CUDA events and returns
  the fastest.
* ``tune_batch`` times candidate (k, warps per CTA, tiles per work item)
  configurations of the batched persistent launch on a sample of the
  circuits.

Results are cached in a JSON file (``$HISVSIM_TUNE_CACHE``, default
``~/.cache/hisvsim/autotune.json``) keyed by a workload key and the
precision, so a later run reuses the choice without measuring.
"""
from __future__ import annotations

import json
import os
import time

import torch

CACHE = os.environ.get("HISVSIM_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "hisvsim",
                                                            "autotune.json"))


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key, value):
    d = _load()
    d[key] = value
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def cached(key):
    return _load().get(key)


def cached_k(workload, method, precision):
    v = cached(f"state:{workload}:{precision}")
    if v and v.get("method") == method:
        return v.get("k")
    return None


def _time_apply(st, plan, tc, reps, jit=False, regbits=0):
    st.apply(plan, sync=True, tc=tc, jit=jit, regbits=regbits)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st.stream)
    for _ in range(reps):
        st.apply(plan, tc=tc, jit=jit, regbits=regbits)
    e1.record(st.stream)
    e1.synchronize()
    st.sync()
    return e0.elapsed_time(e1) / reps


# (part builder, k, tensor-core dense parts, tile (0 = default), specialised
# gate-list kernels, register bits per thread (0 = default; specialised only))
STATE_CANDIDATES = (
    ("beam", 6, True, 0, False), ("dagp", 6, True, 0, False), ("beam", 5, True, 0, False),
    ("dfs", 6, True, 0, False), ("beam", 8, True, 0, False), ("beam", 10, False, 0, False),
    ("dagp", 10, False, 0, False), ("beam", 12, False, 0, False), ("dagp", 8, False, 0, False),
    ("beam", 8, False, 0, True), ("beam", 10, False, 0, True), ("beam", 12, False, 0, True),
    ("dagp", 10, False, 0, True), ("beam", 8, True, 0, True), ("beam", 10, False, 13, True),
    ("beam", 8, False, 13, True), ("beam", 9, False, 0, True), ("beam", 11, False, 13, True),
    ("beam", 9, False, 0, True, 4), ("beam", 10, False, 13, True, 4), ("beam", 9, False, 13, True, 4),
    # tc = 2: two consecutive dense parts per pass where they fit one 13-qubit tile
    ("beam", 6, 2, 0, False), ("dagp", 6, 2, 0, False), ("beam", 5, 2, 0, False),
)
BEAM_WIDTH = 64   # beam builder width for the tuned plans (0.3 s for 2520 gates)


def tune_state(workload, n, gates, precision="c64", candidates=STATE_CANDIDATES, reps=1, state=None,
               use_cache=True, log=None):
    """Fastest (method, k, tc, tile) for this circuit; tc is ignored for
    complex128. Returns a dict with the choice and every measurement."""
    from . import api
    key = f"state:{workload}:{precision}"
    if use_cache and cached(key):
        return cached(key)
    own = state is None
    st = state if state is not None else api.State(n, precision)
    trials = []
    for cand in candidates:
        method, k, tc, tile = cand[:4]
        jit = cand[4] if len(cand) > 4 else False
        regbits = cand[5] if len(cand) > 5 else 0
        if precision != "c64" and tc:
            continue
        if k > n:
            continue
        t0 = time.perf_counter()
        plan = api.Plan(gates, n, method, k, dfs_trials=BEAM_WIDTH if method == "beam" else 16)
        plan_s = time.perf_counter() - t0
        compile_s = 0.0
        try:
            if tile:
                from . import _native as N
                N.check(N.lib.sv_set_tile(st.h, tile))
            if jit:
                compile_s = plan.specialise(precision, tile, tc=tc, regbits=regbits)
            ms = _time_apply(st, plan, tc, reps, jit=jit, regbits=regbits)
            stats = plan.stats(precision, tile, tc=tc, regbits=regbits)
        except Exception as e:   # a configuration the library rejects (tile too small, no NVRTC)
            if log:
                log(f"tune: skip {method} k={k} tc={tc} tile={tile} jit={jit}: {e}")
            plan.close()
            continue
        finally:
            if tile:
                from . import _native as N
                N.lib.sv_set_tile(st.h, 0)
        trials.append({"method": method, "k": k, "tc": tc, "tile": tile, "jit": jit, "regbits": regbits,
                       "ms": round(ms, 3),
                       "passes": stats["passes"], "plan_s": round(plan_s, 3), "compile_s": round(compile_s, 2)})
        plan.close()
    if own:
        st.close()
    if not trials:
        raise RuntimeError("no candidate configuration ran")
    best = min(trials, key=lambda r: r["ms"])
    out = dict(best)
    out["trials"] = trials
    _store(key, out)
    return out


BATCH_CANDIDATES = tuple((k, w, c) for k in (8, 9) for w in (4, 8) for c in (2, 4, 8))


def tune_batch(workload, circuits, method="dfs", candidates=BATCH_CANDIDATES, sample=512, use_cache=True,
               dense_min_qubits=0, methods=None):
    """Fastest (part builder, k, warps per CTA, tiles per item) of the batched
    launch on the first ``sample`` circuits; ``methods`` lists the builders
    tried for the gate-list circuits (default: just ``method``). With
    dense_min_qubits > 0 the larger circuits run on the batched tensor-core
    kernel in the same launch (beam-search plans) and the tuned choice
    applies to the others."""
    from .batch import Batch
    methods = tuple(methods) if methods else (method,)
    key = f"batch:{workload}:c64:dense{dense_min_qubits}:{'+'.join(methods)}"
    if use_cache and cached(key):
        return cached(key)
    sub = circuits[:sample]
    trials = []
    built = {}
    for m in methods:
        for k, w, c in candidates:
            if (m, k) not in built:
                built[(m, k)] = Batch(sub, method=m, k=k, dense_min_qubits=dense_min_qubits)
            b = built[(m, k)]
            b.configure(w, c)
            b.run(sync=True)   # builds and captures
            b.reset()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(b.stream)
            b.run()
            e1.record(b.stream)
            e1.synchronize()
            b.sync()
            trials.append({"method": m, "k": k, "warps": w, "chunk": c, "ms": round(e0.elapsed_time(e1), 3)})
    for b in built.values():
        b.close()
    best = min(trials, key=lambda r: r["ms"])
    out = dict(best)
    out["trials"] = trials
    _store(key, out)
    return out


# Cost model of one apply, from measurements on GB300 (complex64): a part
# pass moves 2 x 8 x 2^n bytes at ~6.3 TB/s on any kernel; the gate-list
# interpreter adds ~2.6e-13 s per op and amplitude (28-qubit layered circuit
# at k = 10: 245 ms for 91 passes and 2420 ops; 33-qubit QFT: 1656 ms for 31
# passes and 475 ops), the plan's specialised kernels ~1.6e-14 s (beam k = 8:
# 74 ms for 94 passes and ~2400 ops).
PASS_BYTES_PER_S = 6.3e12
OP_S_PER_AMP = 2.6e-13
OP_S_PER_AMP_JIT = 1.6e-14


def estimate_s(n, stats, tc, jit=False):
    """Estimated seconds of one apply of a plan with these statistics."""
    t = stats["passes"] * 2 * 8 * (1 << n) / PASS_BYTES_PER_S
    if not tc or stats["dense"] < stats["passes"]:
        t += stats["ops"] * (1 << n) * (OP_S_PER_AMP_JIT if jit else OP_S_PER_AMP)
    return t


# (builder, k, tensor-core dense parts, specialised kernels, smallest n)
PLAN_CANDIDATES = (("beam", 6, True, False, 0), ("beam", 10, False, False, 0), ("beam", 8, False, True, 29),
                   ("beam", 10, False, True, 29))


def choose_plan(gates, n, candidates=PLAN_CANDIDATES):
    """Build each candidate plan and keep the one the cost model rates
    fastest; returns (plan, tc, estimates, jit). Specialised candidates
    (compiled for the plan with NVRTC, ~0.3-3 s of host time, at its first
    apply or by Plan.specialise) are tried only for states large enough that
    their passes save more than the compilation costs. The other plans are
    closed."""
    from . import api
    best = None
    est = []
    for cand in candidates:
        method, k, tc = cand[:3]
        jit = cand[3] if len(cand) > 3 else False
        if len(cand) > 4 and n < cand[4]:
            continue
        plan = api.Plan(gates, n, method, min(k, n), dfs_trials=16)
        e = estimate_s(n, plan.stats("c64", 0, tc=tc), tc, jit)
        est.append({"method": method, "k": k, "tc": tc, "jit": jit, "est_s": e})
        if best is None or e < best[2]:
            if best is not None:
                best[0].close()
            best = (plan, tc, e, jit)
        else:
            plan.close()
    plan, tc, _, jit = best
    return plan, tc, est, jit
