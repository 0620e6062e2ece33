"""Serving loop with continuous batching over the C ABI.

Requests (a circuit on n qubits and an arrival time) are admitted in arrival
order once their state fits: 8 * 2^n bytes against a device byte budget and
a free slot. Admitted states stay on the device until their result is taken.

* Small circuits (n <= small_n) are collected into micro-batches: whenever
  the batched kernel is idle, every admitted small request that has not
  started runs in one batched persistent launch (sv_batch_*), so requests
  that arrived while the previous batch was on the GPU join the next one.
* Large circuits get their own state and CUDA stream and run their part
  passes (sv_apply_parts) beside the batch; at most ``large_running`` of
  them at a time, in arrival order (each pass fills the GPU, so sharing it
  among many large requests only stretches all their latencies). The batch
  stream has the higher priority, so small requests are not queued behind
  the passes of large ones. Each large request runs the plan the cost model
  of ``autotune.choose_plan`` rates fastest: the tensor-core dense plan
  (beam-search parts, k = 6) or the gate-list plan (beam-search parts,
  k = 10; faster for circuits made mostly of diagonal gates such as the QFT).
  With ``tc=False`` large requests use ``method_large`` / ``k_large`` on the
  gate-list kernel. Small requests are planned with the beam builder (k = 9,
  width 4) by default.

A request's result is its probability vector summary: the norm (FP64
accumulation on the device), the probability of |0...0> and the most likely
basis state with its probability; the full state can be kept for checks.
Latency = completion time - arrival time. ``mode="gatewise"`` serves the same
stream with one plain pass per gate for every request (no batching), the
comparison the paper's per-gate simulators correspond to.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import time

import numpy as np
import torch

from . import _native as N
from . import autotune
from .api import Plan, State
from .batch import Batch


@dataclasses.dataclass
class Request:
    rid: int
    n: int
    gates: list
    arrival: float
    family: str = ""


@dataclasses.dataclass
class Result:
    rid: int
    n: int
    arrival: float
    start: float
    done: float
    norm: float
    p0: float
    argmax: int
    pmax: float
    state: object = None

    @property
    def latency(self):
        return self.done - self.arrival


def _summary(probs: torch.Tensor):
    p0 = float(probs[0].item())
    am = int(torch.argmax(probs).item())
    return p0, am, float(probs[am].item())


class Server:
    def __init__(self, budget_bytes=170e9, max_slots=4096, small_n=20, batch_max=512, k_small=9,
                 k_large=6, tc=True, method_small="beam", method_large="dagp", mode="parts",
                 keep_states=False, planners=8, large_running=2):
        self.budget = float(budget_bytes)
        self.max_slots = max_slots
        self.small_n = small_n
        self.batch_max = batch_max
        self.k_small = k_small
        self.k_large = k_large
        self.tc = tc
        self.method_small = method_small
        self.method_large = method_large
        self.mode = mode
        self.keep = keep_states
        self.large_running = large_running
        self.pool = cf.ThreadPoolExecutor(max_workers=planners)
        self.streams = [torch.cuda.Stream() for _ in range(max(1, large_running))]
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
        self.batch_stream = torch.cuda.Stream(priority=hi)

    @staticmethod
    def state_bytes(n):
        return 8 * (1 << n)

    def run(self, requests, time_scale=1.0, log=None):
        """Serve the requests (sorted by arrival); arrival times are replayed
        on the wall clock scaled by time_scale. Returns (results, stats)."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending = collections.deque()
        small_wait = []                    # admitted small requests not started
        large_wait = collections.deque()   # admitted large requests not started
        running_large = []                 # (req, state, plan, event, start)
        batch_run = None                   # (reqs, batch, event, start)
        used = 0.0
        slots = 0
        results = []
        i = 0
        t0 = time.perf_counter()
        s_i = 0
        planned = {}
        host = {"plan_wait_s": 0.0, "batch_build_s": 0.0, "batches": 0, "batched_requests": 0, "large_tc": 0}
        batch_times, batch_sizes, large_times = [], [], []   # launch -> results, per micro-batch / large request

        def now():
            return (time.perf_counter() - t0) / time_scale

        def plan_future(r, method, k, small):
            if self.mode != "parts":
                return self.pool.submit(lambda: (Plan(r.gates, r.n, "none", min(k, r.n)), False))
            if small or not self.tc:
                return self.pool.submit(lambda: (Plan(r.gates, r.n, method, min(k, r.n),
                                                      dfs_trials=4 if method == "beam" else 16), False))
            return self.pool.submit(lambda: autotune.choose_plan(r.gates, r.n)[:2])

        while i < len(reqs) or pending or small_wait or large_wait or running_large or batch_run:
            t = now()
            while i < len(reqs) and reqs[i].arrival <= t:
                r = reqs[i]
                pending.append(r)
                small = r.n <= self.small_n and self.mode == "parts"
                planned[r.rid] = plan_future(r, self.method_small if small else self.method_large,
                                             self.k_small if small else self.k_large, small)
                i += 1
            # admission in arrival order
            while pending:
                r = pending[0]
                b = self.state_bytes(r.n)
                if slots >= self.max_slots or used + b > self.budget:
                    break
                pending.popleft()
                used += b
                slots += 1
                if r.n <= self.small_n and self.mode == "parts":
                    small_wait.append(r)
                else:
                    large_wait.append(r)
            # large requests start in arrival order as running slots free up
            while large_wait and len(running_large) < max(1, self.large_running):
                r = large_wait.popleft()
                st = State(r.n, "c64", stream=self.streams[s_i % len(self.streams)])
                s_i += 1
                w0 = time.perf_counter()
                plan, tc = planned.pop(r.rid).result()
                host["plan_wait_s"] += time.perf_counter() - w0
                host["large_tc"] += int(tc)
                start = now()
                st.apply(plan, gatewise=self.mode != "parts", tc=tc)
                ev = torch.cuda.Event()
                ev.record(st.stream)
                running_large.append((r, st, plan, ev, start))
            # the batched kernel takes every waiting small request when idle
            if batch_run is None and small_wait:
                take, small_wait = small_wait[: self.batch_max], small_wait[self.batch_max:]
                w0 = time.perf_counter()
                plans = [planned.pop(r.rid).result()[0] for r in take]
                w1 = time.perf_counter()
                host["plan_wait_s"] += w1 - w0
                start = now()
                b = Batch.from_plans([(r.n, p) for r, p in zip(take, plans)], stream=self.batch_stream)
                b.run()
                host["batch_build_s"] += time.perf_counter() - w1
                host["batches"] += 1
                host["batched_requests"] += len(take)
                ev = torch.cuda.Event()
                ev.record(b.stream)
                batch_run = (take, b, ev, start)
            # completions
            still = []
            for r, st, plan, ev, start in running_large:
                if ev.query():
                    st.sync()
                    probs = torch.empty(1 << r.n, dtype=torch.float32, device="cuda")
                    with torch.cuda.stream(st.stream):
                        norm = st.probs(probs)
                        p0, am, pm = _summary(probs)
                    res = Result(r.rid, r.n, r.arrival, start, now(), norm, p0, am, pm,
                                 st.copy_to_host() if self.keep else None)
                    results.append(res)
                    large_times.append(res.done - start)
                    st.close()
                    plan.close()
                    used -= self.state_bytes(r.n)
                    slots -= 1
                else:
                    still.append((r, st, plan, ev, start))
            running_large = still
            if batch_run is not None and batch_run[2].query():
                take, b, ev, start = batch_run
                b.sync()
                probs, norms = b.probs()
                torch.cuda.current_stream().wait_stream(b.stream)
                done_t = now()
                batch_times.append(done_t - start)
                batch_sizes.append(len(take))
                for j, r in enumerate(take):
                    p = probs[int(b.offsets[j]):int(b.offsets[j + 1])]
                    p0, am, pm = _summary(p)
                    results.append(Result(r.rid, r.n, r.arrival, start, done_t, float(norms[j]), p0, am, pm,
                                          b.state_host(j) if self.keep else None))
                    used -= self.state_bytes(r.n)
                    slots -= 1
                b.close()
                batch_run = None
            if not (running_large or batch_run) and i < len(reqs) and not pending and not small_wait \
                    and not large_wait:
                wait = reqs[i].arrival - now()
                if wait > 0:
                    time.sleep(min(wait * time_scale, 0.01))
            elif running_large or batch_run:
                time.sleep(0.0002)
        wall = now()
        lat = np.array([r.latency for r in results]) if results else np.zeros(1)
        stats = {"requests": len(results), "wall_s": wall, "circuits_per_s": len(results) / max(wall, 1e-9),
                 "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                 "mean_s": float(lat.mean()), "mode": self.mode, **host}
        # where the latency goes: time from a micro-batch's (large request's)
        # launch to its results, and the micro-batch sizes
        for name, v in (("batch_s", batch_times), ("large_s", large_times)):
            if v:
                stats[name + "_mean"] = round(float(np.mean(v)), 4)
                stats[name + "_max"] = round(float(np.max(v)), 4)
        if batch_sizes:
            stats["batch_size_max"] = int(max(batch_sizes))
        results.sort(key=lambda r: r.rid)
        return results, stats
