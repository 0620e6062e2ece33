"""Serving loop with continuous batching over the C ABI.

Requests (a circuit on n qubits and an arrival time) are admitted once their
state fits: 8 * 2^n bytes against a device byte budget and a free slot.
Admitted states stay on the device until their result is taken.

* Admission. Small requests (n <= small_n) and large ones queue apart, each
  in arrival order. A large request at the head of its queue that does not
  fit waits for memory to free up, without holding back the small requests
  behind it; small and medium (n <= mid_n) requests queue apart too, and
  while a large request waits each class is admitted only within its share
  of the budget (``small_budget``, default 1/8), so they cannot starve it.
* Planning never blocks the loop. Each request's plan is built on a worker
  thread as it arrives (small, medium and large requests on separate pools,
  so no class's plans queue behind another's); a request joins a
  micro-batch, or starts, only once its plan is ready.
* Small requests run in micro-batches on the batched persistent launch
  (sv_batch_*): the circuits of >= 13 qubits on the batched tensor-core
  kernel (beam-search parts of <= 6 qubits), the others on the gate-list
  kernel, in one graph. A builder thread assembles the next micro-batch
  (allocation, program upload, graph capture) from the ready small requests
  while the current one runs, and its graph is launched on the next of two
  batch streams behind the running one, so the GPU goes from one
  micro-batch to the next without a host round trip. Requests that arrive
  meanwhile join the batch after.
* Large requests get their own state and CUDA stream and run their part
  passes (sv_apply_parts) beside the batches, in two lanes: medium ones
  (n <= mid_n, states up to 512 MiB) at most ``mid_running`` at a time, the
  largest at most ``large_running`` at a time (each of their passes fills the
  GPU, so sharing it among many only stretches all their latencies). Stream
  priorities order the lanes: batches first, then medium requests, then the
  largest, so a medium request's passes go between a large one's instead of
  queueing behind it. Each large request runs the plan the cost model of
  ``autotune.choose_plan`` rates fastest: the tensor-core dense plan
  (beam-search parts, k = 6) or the gate-list plan (beam-search parts,
  k = 10); with ``jit_large`` also, for states of 29 qubits and more, the
  plan's specialised kernels (k = 8 or 10), compiled on the planner thread
  (off by default: a compilation takes 1-3 s of host time per request, which
  under a stream of thousands of large requests holds the planners up more
  than the kernels save). With ``tc=False`` large requests use ``method_large`` /
  ``k_large`` on the gate-list kernel.

A request's result is a summary of its probability distribution (Sec. II-A):
the norm (FP64 accumulation on the device), the probability of |0...0> and
the most likely basis state with its probability; large requests get it from
a device reduction that writes no probability vector (sv_measure_summary),
so the only device memory a request holds is its state. The full state can
be kept for checks. Latency = completion time - arrival time.
``mode="gatewise"`` serves the same stream with one plain pass per gate for
every request (no batching), the comparison the paper's per-gate simulators
correspond to.
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

N_CLASSES = ((10, 20), (21, 26), (27, 33))


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
    admitted: float
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


def _pct(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


class Server:
    def __init__(self, budget_bytes=170e9, max_slots=4096, small_n=20, batch_max=512, k_small=9,
                 k_large=6, tc=True, method_small="beam", method_large="dagp", mode="parts",
                 keep_states=False, planners=8, large_planners=4, large_running=2, dense_min_qubits=13,
                 small_budget=None, mid_n=26, mid_running=4, mid_planners=4, jit_large=False):
        self.budget = float(budget_bytes)
        self.small_budget = float(small_budget) if small_budget is not None else self.budget / 8
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
        self.large_running = max(1, large_running)
        self.mid_n = mid_n
        self.mid_running = max(1, mid_running)
        self.dense_min = dense_min_qubits if (tc and mode == "parts") else 0
        self.pool = cf.ThreadPoolExecutor(max_workers=planners)
        self.pool_large = cf.ThreadPoolExecutor(max_workers=large_planners)
        self.pool_mid = cf.ThreadPoolExecutor(max_workers=mid_planners)
        self.jit_large = jit_large
        self.builder = cf.ThreadPoolExecutor(max_workers=1)
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
        mid = max(hi, lo - 1) if hi < lo else lo   # one step above the lowest priority
        self.streams = [torch.cuda.Stream(priority=lo) for _ in range(self.large_running)]
        self.mid_streams = [torch.cuda.Stream(priority=mid) for _ in range(self.mid_running)]
        self.batch_streams = [torch.cuda.Stream(priority=hi) for _ in range(2)]

    @staticmethod
    def state_bytes(n):
        return 8 * (1 << n)

    def _small(self, r):
        return r.n <= self.small_n and self.mode == "parts"

    def _plan(self, r):
        """Built on a worker thread: (plan, tc, jit)."""
        if self.mode != "parts":
            return Plan(r.gates, r.n, "none", min(self.k_large, r.n)), False, False
        if self._small(r):
            if self.dense_min and r.n >= self.dense_min:
                return Plan(r.gates, r.n, "beam", 6, dfs_trials=4), True, False
            return Plan(r.gates, r.n, self.method_small, min(self.k_small, r.n),
                        dfs_trials=4 if self.method_small == "beam" else 16), False, False
        if not self.tc:
            return Plan(r.gates, r.n, self.method_large, min(self.k_large, r.n)), False, False
        cands = autotune.PLAN_CANDIDATES if self.jit_large else tuple(
            c for c in autotune.PLAN_CANDIDATES if not (len(c) > 3 and c[3]))
        plan, tc, _, jit = autotune.choose_plan(r.gates, r.n, candidates=cands)
        if jit:
            plan.specialise("c64", 0, tc=tc)   # compiled here, on the planner thread
        return plan, tc, jit

    def _build_batch(self, take, plans, stream):
        """Built on the builder thread: the micro-batch with its graph captured."""
        t0 = time.perf_counter()
        b = Batch.from_plans([(r.n, p) for r, p in zip(take, plans)], stream=stream,
                             dense_min_qubits=self.dense_min)
        b.prepare()
        return b, time.perf_counter() - t0

    @staticmethod
    def _new_state(n, stream):
        try:
            return State(n, "c64", stream=stream)
        except (torch.cuda.OutOfMemoryError, N.SvError) as e:
            if isinstance(e, N.SvError) and e.status != N.SV_ERR_OOM:
                raise
            # blocks of other sizes cached by torch's allocator: return them and retry
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            return State(n, "c64", stream=stream)

    def run(self, requests, time_scale=1.0, log=None):
        """Serve the requests (sorted by arrival); arrival times are replayed
        on the wall clock scaled by time_scale. Returns (results, stats)."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        pend_small = collections.deque()      # arrived, not admitted (arrival order)
        pend_mid = collections.deque()
        pend_large = collections.deque()
        small_wait = collections.deque()      # admitted small requests not in a batch
        large_wait = []                       # admitted large requests not started
        running_large = []                    # (req, state, plan, event, start)
        building = None                       # (take, future) of the next micro-batch
        in_flight = collections.deque()       # launched micro-batches: (take, batch, event, start)
        futures = {}
        admitted_at = {}
        used = 0.0
        class_used = [0.0, 0.0]               # small, medium
        slots = 0
        results = []
        i = 0
        bsi = 0                               # next batch stream
        lsi = 0                               # next large-request stream
        msi = 0                               # next medium-request stream
        host = {"batch_build_s": 0.0, "batches": 0, "batched_requests": 0, "large_tc": 0, "large_jit": 0,
                "admission_stalls": 0, "peak_used_bytes": 0.0}
        batch_times, batch_sizes, large_times = [], [], []
        stalled = False
        t0 = time.perf_counter()

        def now():
            return (time.perf_counter() - t0) / time_scale

        def finish(r, start, done, norm, p0, am, pm, state):
            nonlocal used, slots
            results.append(Result(r.rid, r.n, r.arrival, admitted_at.pop(r.rid), start, done, norm, p0, am, pm,
                                  state))
            used -= self.state_bytes(r.n)
            if self._small(r):
                class_used[0] -= self.state_bytes(r.n)
            elif r.n <= self.mid_n:
                class_used[1] -= self.state_bytes(r.n)
            slots -= 1

        while (i < len(reqs) or pend_small or pend_mid or pend_large or small_wait or large_wait or running_large
               or building or in_flight):
            t = now()
            while i < len(reqs) and reqs[i].arrival <= t:
                r = reqs[i]
                small = self._small(r)
                pool = self.pool if small else self.pool_mid if r.n <= self.mid_n else self.pool_large
                futures[r.rid] = pool.submit(self._plan, r)
                (pend_small if small else pend_mid if r.n <= self.mid_n else pend_large).append(r)
                i += 1
            # admission: large requests in arrival order while the head fits
            while pend_large:
                r = pend_large[0]
                b = self.state_bytes(r.n)
                if slots >= self.max_slots or used + b > self.budget:
                    if not stalled:
                        host["admission_stalls"] += 1
                    stalled = True
                    break
                stalled = False
                pend_large.popleft()
                used += b
                slots += 1
                admitted_at[r.rid] = now()
                large_wait.append(r)
            # small and medium requests in arrival order beside them; while a
            # large request waits, each class stays within its share of the
            # budget (small_budget), so the memory finished large requests
            # free reaches the waiting head
            for pend, dest in ((pend_small, small_wait), (pend_mid, large_wait)):
                while pend:
                    r = pend[0]
                    b = self.state_bytes(r.n)
                    cls = 0 if dest is small_wait else 1
                    if (slots >= self.max_slots or used + b > self.budget
                            or (pend_large and class_used[cls] + b > self.small_budget)):
                        break
                    pend.popleft()
                    used += b
                    class_used[cls] += b
                    slots += 1
                    admitted_at[r.rid] = now()
                    dest.append(r)
            host["peak_used_bytes"] = max(host["peak_used_bytes"], used)
            # large requests start as running slots of their lane free up, once
            # planned: medium ones (n <= mid_n) on their own higher-priority
            # streams, so they do not queue behind the largest states
            j = 0
            while j < len(large_wait):
                r = large_wait[j]
                is_mid = r.n <= self.mid_n
                lane_busy = sum((x[0].n <= self.mid_n) == is_mid for x in running_large)
                if lane_busy >= (self.mid_running if is_mid else self.large_running) or not futures[r.rid].done():
                    j += 1
                    continue
                large_wait.pop(j)
                plan, tc, jit = futures.pop(r.rid).result()
                host["large_tc"] += int(tc)
                host["large_jit"] += int(jit)
                if is_mid:
                    stream = self.mid_streams[msi % len(self.mid_streams)]
                    msi += 1
                else:
                    stream = self.streams[lsi % len(self.streams)]
                    lsi += 1
                st = self._new_state(r.n, stream)
                start = now()
                st.apply(plan, gatewise=self.mode != "parts", tc=tc, jit=jit)
                ev = torch.cuda.Event()
                ev.record(st.stream)
                running_large.append((r, st, plan, ev, start))
            # the next micro-batch: every admitted small request whose plan is ready
            if building is None and small_wait and len(in_flight) < 2:
                take = []
                rest = collections.deque()
                while small_wait:
                    r = small_wait.popleft()
                    if len(take) < self.batch_max and futures[r.rid].done():
                        take.append(r)
                    else:
                        rest.append(r)
                small_wait = rest
                if take:
                    plans = [futures.pop(r.rid).result()[0] for r in take]
                    stream = self.batch_streams[bsi % 2]
                    bsi += 1
                    building = (take, self.builder.submit(self._build_batch, take, plans, stream))
            if building is not None and building[1].done() and len(in_flight) < 2:
                take, fut = building
                building = None
                b, build_s = fut.result()
                host["batch_build_s"] += build_s
                host["batches"] += 1
                host["batched_requests"] += len(take)
                if in_flight:
                    b.stream.wait_event(in_flight[-1][2])   # runs right after the batch in flight
                b.run()
                ev = torch.cuda.Event()
                ev.record(b.stream)
                in_flight.append((take, b, ev, now()))
            # completions
            still = []
            for r, st, plan, ev, start in running_large:
                if ev.query():
                    norm, p0, am, pm = st.summary()
                    done = now()
                    finish(r, start, done, norm, p0, am, pm, st.copy_to_host() if self.keep else None)
                    large_times.append(done - start)
                    st.close()
                    plan.close()
                else:
                    still.append((r, st, plan, ev, start))
            running_large = still
            if in_flight and in_flight[0][2].query():
                take, b, ev, start = in_flight.popleft()
                b.sync()
                probs, norms = b.probs()
                ph = probs.cpu().numpy()
                done = now()
                batch_times.append(done - start)
                batch_sizes.append(len(take))
                for j, r in enumerate(take):
                    p = ph[int(b.offsets[j]):int(b.offsets[j + 1])]
                    am = int(np.argmax(p))
                    finish(r, start, done, float(norms[j]), float(p[0]), am, float(p[am]),
                           b.state_host(j) if self.keep else None)
                b.close()
            idle = not (running_large or building or in_flight)
            if idle and i < len(reqs) and not (pend_small or pend_mid or pend_large or small_wait or large_wait):
                wait = reqs[i].arrival - now()
                if wait > 0:
                    time.sleep(min(wait * time_scale, 0.01))
            else:
                time.sleep(0.0002)
        wall = now()
        last_arrival = reqs[-1].arrival if reqs else 0.0
        stats = self._stats(results, wall, last_arrival, host, batch_times, batch_sizes, large_times)
        results.sort(key=lambda r: r.rid)
        return results, stats

    def _stats(self, results, wall, last_arrival, host, batch_times, batch_sizes, large_times):
        lat = [r.latency for r in results] or [0.0]
        adm = [r.admitted - r.arrival for r in results] or [0.0]
        stats = {"requests": len(results), "wall_s": wall, "circuits_per_s": len(results) / max(wall, 1e-9),
                 "p50_s": _pct(lat, 50), "p99_s": _pct(lat, 99), "mean_s": float(np.mean(lat)),
                 "drain_s": max(0.0, wall - last_arrival), "admit_wait_p99_s": _pct(adm, 99),
                 "admit_wait_max_s": float(np.max(adm)), "mode": self.mode, **host}
        by_class = {}
        for lo, hi in N_CLASSES:
            v = [r.latency for r in results if lo <= r.n <= hi]
            if v:
                by_class[f"{lo}-{hi}"] = {"requests": len(v), "p50_s": round(_pct(v, 50), 4),
                                          "p99_s": round(_pct(v, 99), 4), "max_s": round(max(v), 4)}
        stats["by_n"] = by_class
        # where the latency goes: launch -> results per micro-batch and large request
        for name, v in (("batch_s", batch_times), ("large_s", large_times)):
            if v:
                stats[name + "_mean"] = round(float(np.mean(v)), 4)
                stats[name + "_max"] = round(float(np.max(v)), 4)
        if batch_sizes:
            stats["batch_size_max"] = int(max(batch_sizes))
            stats["batch_size_mean"] = round(float(np.mean(batch_sizes)), 1)
        return stats

    def close(self):
        for p in (self.pool, self.pool_mid, self.pool_large, self.builder):
            p.shutdown(wait=True)
