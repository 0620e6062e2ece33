"""Benchmark of the hierarchical state-vector hot path on GB300.

One step = every part pass of the 28-qubit random layered circuit (depth 60,
H/RX/RZ on every qubit then CX/CZ on a random disjoint pairing; 2520 gates)
applied to a complex64 state resident in HBM, through the C ABI
(sv_apply_parts). The metric is the part passes' algorithmic HBM traffic
(2 x state bytes per pass) per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0. Under torchrun each rank runs an independent
replica on its own GPU (the path has no exchange step on one GPU per state);
value = all ranks' bytes / max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "state-vector part passes GB/s (HBM traffic of the passes / time)"
UNIT = "GB/s"
DTYPE_TC = ("c64 state; split-BF16 x3 tensor-core products, FP32 accumulate in TMEM, per-pass rescale "
            "to the input norm")
DTYPE_FP32 = "c64 state; FP32 arithmetic"
WORKLOAD = ("random layered circuit, 28 qubits, depth 60 (H/RX/RZ on every qubit, then CX/CZ on a "
            "random disjoint pairing; 2520 gates, seed 2), complex64 state, part-fused passes")



def workload_text(n, n_gates):
    """The workload line for the layered circuit on n qubits (28 by default)."""
    return WORKLOAD.replace("28 qubits", f"{n} qubits").replace("2520 gates", f"{n_gates} gates")

def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--method", default="dagp", choices=["nat", "dfs", "dagp", "beam"],
                    help="part builder with --k (the reference arm's oracle has nat, dfs, dagp; beam maps to dagp)")
    ap.add_argument("--k", type=int, default=0, help="part qubit limit (0: autotuned default)")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--tc", type=int, default=0, help="with --k: run parts of <= 6 qubits on the tensor cores "
                    "(2: two consecutive such parts per pass where they fit one 13-qubit tile)")
    ap.add_argument("--jit", type=int, default=0, help="with --k: gate-list parts on the plan's specialised kernels")
    ap.add_argument("--regbits", type=int, default=0, help="with --jit: register bits per thread (0 = default)")
    ap.add_argument("--no-grid", action="store_true", help="skip the builder x k grid and the complex128 line")
    ap.add_argument("--n", type=int, default=28)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-e2e-child", action="store_true",
                    help="measure the end-to-end loop only in this process")
    ap.add_argument("--e2e-only", action="store_true",
                    help="run only the end-to-end loop for the plan given by --method/--k/--tc/--jit/--regbits/--tile")
    ap.add_argument("--e2e-states", type=int, default=3,
                    help="states in turn in the end-to-end loop (copies of one overlap the others' passes)")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 4096-circuit batched launch")
    ap.add_argument("--batch-circuits", type=int, default=4096,
                    help="circuits of the batch section (a smaller batch for profiling)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving section")
    ap.add_argument("--serving-window", type=float, default=3.0,
                    help="seconds of the request stream's arrivals served in the serving section")
    ap.add_argument("--serving-only", action="store_true",
                    help="only the serving section (what the benchmark runs in a child process), one JSON line")
    ap.add_argument("--serving-jit-large", action="store_true",
                    help="with --serving-full: specialised kernels for requests of >= 29 qubits")
    ap.add_argument("--serving-full", action="store_true",
                    help="serve the whole 20000-request stream (60 s of arrivals, then drain; minutes), "
                         "one JSON line, then exit")
    ap.add_argument("--partition-quality", action="store_true",
                    help="CPU only: part counts of Nat, DFS and dagP against the exact optimum on small "
                         "circuits (one JSON line), then exit")
    ap.add_argument("--oracle-report", action="store_true",
                    help="with --impl reference: time the oracle in both modes, 1 thread and all cores, on the "
                         "configurations' workloads (bounded prefixes, scaled), one JSON line each")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = {
    "k_dense6": ("dense.cu", "dense.hpp", "dense_common.cuh", "planner.cpp"),
    "k_dense6_pair": ("dense_pair.cu", "dense.hpp", "dense_common.cuh", "planner.cpp"),
    "k_part": ("kernels.cu", "ops.cuh", "ops_core.cuh", "program.hpp", "planner.cpp"),
    "hisv_part": ("jit.cpp", "jit_prelude.cuh", "ops_core.cuh", "program.hpp", "planner.cpp"),
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2205_06973_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel, workload_key):
    """DRAM bytes per launch of the kernel from the committed ncu summary
    (profiles/traffic.txt), if it was taken on the current kernel source
    (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    cur = kernel_source_hash(kernel)
    with open(path) as f:
        for line in f:
            if line.lstrip().startswith("#"):
                continue
            parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
            if (parts.get("kernel") == kernel and parts.get("source") == cur
                    and parts.get("workload") == workload_key):
                try:
                    return float(parts["bytes_per_launch"])
                except (KeyError, ValueError):
                    return None
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x, device):
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline_oracle(n, gates, pog, n_parts, max_parts, budget_s=20.0):
    """The oracle's Algorithm 1 mode (complex128, OpenMP on the host cores) on
    the first parts of the same plan, until about budget_s of CPU time."""
    import numpy as np
    from oracle import sim
    pog = np.asarray(pog, dtype=np.uint32)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    done = 0
    t0 = time.perf_counter()
    while done < min(max_parts, n_parts):
        sel = pog == done
        sub = [g for g, s in zip(gates, sel) if s]
        psi = sim.run_alg1(n, sub, [0] * len(sub), 1, psi)
        done += 1
        el = time.perf_counter() - t0
        if el + el / done > budget_s:   # the next part would end past the budget
            break
    dt = time.perf_counter() - t0
    bytes_per_pass = 2 * 16 * (1 << n)
    return {"value": bytes_per_pass * done / dt / 1e9, "unit": UNIT, "cores": sim.num_threads(),
            "kind": "oracle",
            "sample": f"first {done} of {n_parts} parts of the same plan, Algorithm 1 mode, complex128 "
                      f"(32 B/amplitude per pass), {dt:.1f} s"}


def batch_section(count=4096):
    """4096 parameterised circuits (10-20 qubits, RY/RZ layers + CX ladder,
    depth 10-50) in one graph-captured launch pair: the circuits of >= 13
    qubits as dense 64x64 tensor-core passes (beam-search parts of <= 6
    qubits) in the batched tensor-core kernel, the others on the gate-list
    kernel, whose part builder (DFS or beam), k, warps per CTA and tiles per
    work item the autotuner picks on 512 of them."""
    import numpy as np
    import torch
    import synth
    from paper_2205_06973_gb300 import autotune
    from paper_2205_06973_gb300.batch import Batch
    circs = synth.batch_circuits(count)
    t0 = time.perf_counter()
    choice = autotune.tune_batch(f"param{count}", circs, methods=("dfs", "beam"), use_cache=False,
                                 dense_min_qubits=13)
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = Batch(circs, method=choice["method"], k=choice["k"], warps_per_cta=choice["warps"],
              tiles_per_item=choice["chunk"], dense_min_qubits=13)
    plan_s = time.perf_counter() - t0
    b.run(sync=True)            # builds the work list and captures the graph
    b.reset()
    b.run(sync=True)
    bytes_all = 0
    for (n, _), p in zip(circs, b.plans):
        _, parts = p.export()
        bytes_all += parts * 2 * 8 * (1 << n)
    reps = 3
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    for _ in range(reps):
        b.run()
    e1.record(b.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    b.reset()
    b.run(sync=True)
    _, norms = b.probs()
    info = b.info()
    b.close()
    return {"workload": f"{count} parameterised circuits, 10-20 qubits (uniform), RY/RZ layers + CX ladder, "
                        "depth 10-50, complex64, one graph: circuits of >= 13 qubits on the batched "
                        "tensor-core kernel (beam-search parts of <= 6 qubits as 64x64 split-BF16 passes, work in "
                        "L2-sized circuit groups), the rest on the gate-list kernel",
            "circuits_per_s": round(count / ms * 1e3, 1), "ms_per_launch": round(ms, 2),
            "GBs": round(bytes_all / ms / 1e6, 1), "bytes_per_launch": bytes_all,
            "autotune": {k: choice[k] for k in ("method", "k", "warps", "chunk")}, "tune_s": round(tune_s, 1),
            "plan_s": round(plan_s, 1), "parts": info.get("parts"), "items": info.get("items"),
            "dense_circuits": info.get("dense_circuits"), "dense_passes": info.get("dense_passes"),
            "dense_items": info.get("dense_items"),
            "norm_min": float(np.min(norms)), "norm_max": float(np.max(norms))}


def _serving_requests(count, window_s=None, max_n=33):
    """The serving stream (seed 5: 20000 Poisson arrivals over 60 s, 10-33
    qubits with 80 % <= 20, three families): its first ``count`` requests of at
    most max_n qubits, or every request arriving in the first window_s
    seconds."""
    import synth
    from paper_2205_06973_gb300.serving import Request
    arr = synth.serving_arrivals(20000, 60.0, seed=5)
    reqs, i = [], 0
    while i < len(arr) and (window_s is None or arr[i] <= window_s) and (window_s is not None or len(reqs) < count):
        n, fam, g = synth.serving_request(i, seed=5)
        if n <= max_n:
            reqs.append(Request(len(reqs), n, g, arr[i], fam))
        i += 1
    return reqs


def _serving_stats(st):
    return {k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items() if k != "mode"}


def serving_section(window_s=3.0):
    """The serving loop on the request stream: (1) every request arriving in
    the stream's first window_s seconds, all qubit counts (10-33, states up to
    64 GiB, admission by 8 * 2^n bytes against 170 GB), part-fused, served to
    the end (drain); (2) the first 300 requests of at most 26 qubits,
    part-fused and gate by gate (gate by gate takes minutes per 33-qubit
    request, so the comparison runs on this sample)."""
    from paper_2205_06973_gb300.serving import Server
    win = _serving_requests(None, window_s=window_s)
    srv = Server(budget_bytes=170e9)
    _, st = srv.run(win)
    srv.close()
    out = {"stream": {"workload": f"every request of the first {window_s:g} s of arrivals of the 20000-request "
                                  "stream (seed 5), 10-33 qubits, arrival times replayed, served until drained",
                      "n_requests": len(win), "n_min": min(r.n for r in win), "n_max": max(r.n for r in win),
                      "n_27_33": sum(r.n >= 27 for r in win), **_serving_stats(st)}}
    sample = _serving_requests(300, max_n=26)
    out["sample"] = {"workload": "first 300 requests with n <= 26 of the same stream, arrival times replayed",
                     "n_large": sum(r.n > 20 for r in sample)}
    for mode in ("parts", "gatewise"):
        srv = Server(budget_bytes=170e9, mode=mode)
        _, st = srv.run(sample)
        srv.close()
        out["sample"][mode] = _serving_stats(st)
    sp = out["sample"]
    sp["throughput_vs_gate_by_gate"] = round(sp["parts"]["circuits_per_s"] / sp["gatewise"]["circuits_per_s"], 2)
    sp["p99_vs_gate_by_gate"] = round(sp["gatewise"]["p99_s"] / sp["parts"]["p99_s"], 2)
    return out



def e2e_loop(n, plan, tc, jit, regbits, tile, S, host_in, host_out, ws, dev, bytes_per_step, reps=12,
             states=None):
    """The end-to-end metric through the C ABI: every step uploads its input
    from pinned host memory (sv_upload), applies the plan (sv_apply_parts)
    and downloads its result (sv_download). S states on S streams are used
    in turn, so a step's upload and download overlap the other states'
    passes; each step's passes wait for the previous step's passes (an
    event), so the states take turns on the SMs instead of sharing them and
    the copies leave the compute timeline. A state is reused only after its
    download of S steps back has reached host memory, which gives a
    download and the next upload S - 1 steps of passes to hide in (the host
    link's rate varies from box to box and under other jobs' host memory
    traffic). ``states``: S states to use (each on its own stream; kept
    open), else S are allocated here and closed at the end."""
    import torch
    from paper_2205_06973_gb300 import api
    own = states is None
    sts = [api.State(n, "c64", stream=torch.cuda.Stream(), tile=tile) for _ in range(S)] if own else states
    if not own:
        for x in sts:
            x.set_tile(tile)

    def step(i, last):
        x = sts[i % S]
        if i >= S:
            x.sync()          # its result of step i - S has reached host memory
        x.upload(host_in)
        if last is not None:
            x.stream.wait_event(last)
        x.apply(plan, tc=tc, jit=jit, regbits=regbits)
        done = torch.cuda.Event()
        done.record(x.stream)
        x.download(host_out[i % S])
        return done

    last = None
    for i in range(S):
        last = step(i, last)
    for x in sts:
        x.sync()
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    last = None
    for i in range(reps):
        last = step(i, last)
    for x in sts:
        x.sync()
    dt = (time.perf_counter() - t0) / reps
    dt = max_over_ranks(ws, dt, dev)
    nbytes = sts[0].nbytes
    if own:
        for x in sts:
            x.close()
    return {"value": round(ws * bytes_per_step / dt / 1e9, 1), "unit": UNIT,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "ms_per_step": round(dt * 1e3, 3), "steps": reps, "states": S,
            "api": f"sv_upload + sv_apply_parts + sv_download (pinned host buffers), {S} states on {S} "
                   "streams taking turns on the SMs, so that a step's copies overlap the other states' passes"}


def pinned_buffers(n, S):
    """The end-to-end loop's pinned host buffers: one input (|0...0>) read by
    every state, one output per state."""
    import torch
    host_in = torch.zeros(1 << n, dtype=torch.complex64).pin_memory()
    host_in[0] = 1.0
    return host_in, [torch.empty(1 << n, dtype=torch.complex64).pin_memory() for _ in range(S)]


def e2e_child(n, method, k, tc, jit, regbits, tile, S):
    """e2e_loop in a fresh process on the same GPU with the given plan
    (bench.py --e2e-only); its e2e object, or {"error": ...}."""
    cmd = [sys.executable, os.path.abspath(__file__), "--e2e-only", "--n", str(n), "--method", method,
           "--k", str(k), "--tc", str(int(tc)), "--jit", str(int(jit)), "--regbits", str(regbits),
           "--tile", str(tile), "--e2e-states", str(S)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    except subprocess.TimeoutExpired:
        return {"error": "fresh-process end-to-end run timed out"}
    for line in reversed(r.stdout.strip().splitlines()):
        if line.startswith("{"):
            try:
                out = json.loads(line)["e2e"]
                out["process"] = "fresh process: loads the tuned plan and runs only this loop"
                return out
            except (ValueError, KeyError):
                break
    return {"error": f"e2e child exited {r.returncode}: " + " | ".join(r.stderr.strip().splitlines()[-3:])}


def run_e2e_only(a):
    """bench.py --e2e-only: the end-to-end loop alone, for the plan given on
    the command line (one JSON line {"e2e": ...})."""
    import torch
    torch.cuda.set_device(0)
    import synth
    from paper_2205_06973_gb300 import api
    from paper_2205_06973_gb300.autotune import BEAM_WIDTH
    n, gates = synth.layered_28q(n=a.n)
    S = max(2, a.e2e_states)
    host_in, host_out = pinned_buffers(n, S)
    plan = api.Plan(gates, n, a.method, a.k, dfs_trials=BEAM_WIDTH if a.method == "beam" else 16)
    tc, jit = int(a.tc), bool(a.jit)
    if jit:
        plan.specialise("c64", a.tile, tc=tc, regbits=a.regbits)
    passes = plan.stats("c64", a.tile, tc=tc, regbits=a.regbits)["passes"]
    e2e = e2e_loop(n, plan, tc, jit, a.regbits, a.tile, S, host_in, host_out, 1, torch.device("cuda", 0),
                   passes * 2 * (8 << n))
    e2e["host_buffers"] = "pinned, allocated at process start"
    plan.close()
    print(json.dumps({"e2e": e2e}), flush=True)

def serving_child(window_s):
    """serving_section in a child process on the same GPU: the serving loop
    runs many streams and host threads at once, and a device fault there
    must not take the benchmark's own context (and its JSON line) down with
    it."""
    cmd = [sys.executable, os.path.abspath(__file__), "--serving-only", "--serving-window", str(window_s)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    for line in reversed(r.stdout.strip().splitlines()):
        if line.startswith("{"):
            try:
                return json.loads(line)["serving"]
            except (ValueError, KeyError):
                break
    return {"error": f"serving child exited {r.returncode}: " + " | ".join(r.stderr.strip().splitlines()[-3:])}


def serving_full(jit_large=False):
    """The whole serving stream (20000 requests over 60 s, 10-33 qubits,
    170 GB budget), part-fused, until drained. One JSON line. jit_large:
    requests of >= 29 qubits may run their plan's specialised kernels
    (compiled on the large-request planner threads)."""
    import torch
    from paper_2205_06973_gb300.serving import Server
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    reqs = _serving_requests(20000)
    gen_s = time.perf_counter() - t0
    clk = ClockSampler(0)
    clk.start()
    srv = Server(budget_bytes=170e9, jit_large=jit_large)
    res, st = srv.run(reqs)
    srv.close()
    clocks = clk.stop()
    print(json.dumps({"serving_full": {"workload": "the 20000-request stream (seed 5): Poisson arrivals over 60 s, "
                                                   "10-33 qubits (80 % <= 20), layered / QFT / parameterised, "
                                                   "complex64, admission by 8 * 2^n bytes against 170 GB",
                                       "jit_large": jit_large, "generate_s": round(gen_s, 1), "clocks": clocks,
                                       "norm_min": min(r.norm for r in res), "norm_max": max(r.norm for r in res),
                                       **_serving_stats(st)}}), flush=True)


# flops per amplitude of each gate kind in the paper's model of a gate pass
# (Sec. III-A: a general one-qubit gate is a 2x2 complex matrix-vector
# product per amplitude pair, 14 flops per amplitude): diagonal gates
# multiply the amplitudes of their non-unit entries (RZ: all; P/S/T: half;
# CP: a quarter), permutations and sign changes cost none
GATE_FLOPS = {"H": 14, "RX": 14, "RY": 14, "X": 0, "Y": 0, "Z": 0, "RZ": 6, "P": 3, "S": 3, "T": 3,
              "CX": 0, "CZ": 0, "SWAP": 0, "CP": 1.5}


def circuit_flops(n, gates):
    return sum(GATE_FLOPS[g[0]] for g in gates) * float(1 << n)


def alu_peaks():
    """Measured FMA rates of the CUDA cores (sv_alu_probe), FLOP/s."""
    import ctypes
    from paper_2205_06973_gb300 import _native as N
    out = {}
    for name, fp64 in (("fp64", 1), ("fp32", 0)):
        v = ctypes.c_double()
        N.check(N.lib.sv_alu_probe(fp64, ctypes.byref(v)))
        out[name] = v.value
    return out


def _timed(st, plan, tc=False, jit=False, reps=2, regbits=0):
    import torch
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


def grid_section(n, gates, st, peak, fp32_peak=None):
    """The paper's three builders at k in {8, 10, 12} on the complex64 state:
    passes, time per step and pass GB/s (fraction of the measured copy
    bandwidth) on the interpreter kernel and on the plan's specialised
    kernels, and the FP32 flops the plan's program executes (sv_plan_flops)
    per second against the measured FP32 FMA rate: the second bound, which
    takes over as the gates per pass grow with k."""
    from paper_2205_06973_gb300 import api
    rows = []
    for method in ("nat", "dfs", "dagp"):
        for k in (8, 10, 12):
            plan = api.Plan(gates, n, method, k)
            passes = plan.stats("c64")["passes"]
            flops = plan.flops("c64")[0]
            row = {"method": method, "k": k, "passes": passes, "executed_fp32_flops": flops}
            for name, jit in (("interpreter", False), ("specialised", True)):
                if jit:
                    row["compile_s"] = round(plan.specialise("c64"), 2)
                ms = _timed(st, plan, jit=jit)
                gbs = passes * 2 * st.nbytes / (ms / 1e3) / 1e9
                row[name] = {"ms": round(ms, 2), "GBs": round(gbs, 1), "frac": round(gbs / peak, 4)}
                if fp32_peak:
                    fl = flops / (ms / 1e3)
                    row[name]["fp32_tflops"] = round(fl / 1e12, 2)
                    row[name]["fp32_frac"] = round(fl / fp32_peak, 4)
            if k == 12:
                # the default tile for k = 12 is 2^13 (the part plus the
                # lowest free qubit); a 2^12 tile holds only the part's own
                # qubits, so a part without the lowest qubits reads runs of
                # one amplitude
                st.set_tile(12)
                plan.specialise("c64", 12)
                ms = _timed(st, plan, jit=True)
                st.set_tile(0)
                gbs = passes * 2 * st.nbytes / (ms / 1e3) / 1e9
                row["specialised_tile12"] = {"ms": round(ms, 2), "GBs": round(gbs, 1), "frac": round(gbs / peak, 4)}
            plan.close()
            rows.append(row)
    return {"workload": "28-qubit layered circuit, complex64 state (2 GiB), gate-list parts",
            "peak_GBs": peak, "fp32_fma_peak_tflops": round(fp32_peak / 1e12, 2) if fp32_peak else None,
            "rows": rows}


def c128_section(n, gates, peak, fp64_peak):
    """The same circuit on a complex128 state (4 GiB, the paper's precision):
    time per step, pass GB/s against the copy bandwidth, and the FP64 flops
    the plan's kernels execute (sv_plan_flops) per second against the
    measured FP64 FMA rate, on the interpreter and on the specialised
    kernels in FP64 and in double-float arithmetic (SV_C128DF: the same
    operations on FP32 pipes, so the rate is FP64-equivalent operations per
    second and may exceed the FP64 peak). The gate model's count
    (GATE_FLOPS, general matrices) is given beside it."""
    from paper_2205_06973_gb300 import api
    st = api.State(n, "c128")
    model = circuit_flops(n, gates)
    rows = []
    sdf = api.State(n, "c128df")
    for method, k, jit, prec in (("dagp", 10, False, "c128"), ("dagp", 10, True, "c128"), ("beam", 10, True, "c128"),
                                 ("beam", 10, True, "c128df"), ("beam", 8, True, "c128df"),
                                 ("dagp", 10, True, "c128df")):
        plan = api.Plan(gates, n, method, k, dfs_trials=16)
        passes = plan.stats("c128")["passes"]
        flops = plan.flops("c128")[0]
        cs = plan.specialise(prec) if jit else 0.0
        ms = _timed(st if prec == "c128" else sdf, plan, jit=jit, reps=1)
        gbs = passes * 2 * st.nbytes / (ms / 1e3) / 1e9
        fl = flops / (ms / 1e3)
        rows.append({"method": method, "k": k, "precision": prec,
                     "arithmetic": "double-float on FP32 pipes" if prec == "c128df" else "FP64",
                     "kernel": "specialised" if jit else "interpreter", "passes": passes,
                     "ms": round(ms, 1), "GBs": round(gbs, 1), "hbm_frac": round(gbs / peak, 4),
                     "executed_fp64_flops": flops, "fp64_tflops": round(fl / 1e12, 3),
                     "fp64_frac": round(fl / fp64_peak, 4), "compile_s": round(cs, 2)})
        plan.close()
    norm = st.probs()
    norm_df = sdf.probs()
    st.close()
    sdf.close()
    return {"workload": "28-qubit layered circuit, complex128 state (4 GiB)", "gate_model_fp64_flops": model,
            "norm_df": norm_df,
            "fp64_peak_tflops": round(fp64_peak / 1e12, 3), "rows": rows, "norm": norm}


def multilevel_section(peak):
    """Multi-level partitioning (Sec. IV-B) against one level, on the
    28-qubit layered circuit (complex64, 2 GiB) and the 33-qubit QFT
    (complex64, 64 GiB): the same first-level parts (HBM passes), their
    register phases from the greedy split (one level) or from a second
    builder under k2 = 5 (two levels), on the specialised kernels."""
    import synth
    from paper_2205_06973_gb300 import api
    out = []
    n33, g33, x33 = synth.qft_basis(33)
    for name, (n, g) in (("layered28", synth.layered_28q()), ("qft33", (n33, g33))):
        st = api.State(n, "c64")
        for m, k in (("dagp", 10), ("beam", 10), ("beam", 12)):
            for inner in (None, ("dagp", 5), ("beam", 5)):
                plan = api.Plan(g, n, m, k, inner=inner)
                stt = plan.stats("c64")
                cs = plan.specialise("c64")
                ms = _timed(st, plan, jit=True, reps=2 if n < 30 else 1)
                gbs = stt["passes"] * 2 * st.nbytes / (ms / 1e3) / 1e9
                out.append({"circuit": name, "method": m, "k": k, "inner": "greedy" if inner is None else
                            f"{inner[0]} k2={inner[1]}", "passes": stt["passes"], "phases": stt["phases"],
                            "ops": stt["ops"], "ms": round(ms, 2), "GBs": round(gbs, 1),
                            "frac": round(gbs / peak, 4), "compile_s": round(cs, 2)})
                plan.close()
        st.close()
    return {"kernel": "specialised gate-list kernels", "rows": out}


def qft33_section(peak):
    """The 33-qubit QFT (577 gates) on the seeded basis state |x> (complex64,
    64 GiB): the tensor-core plan (beam, k = 6) and the specialised
    gate-list plans (beam, k = 10 and 12). (Its amplitudes are checked
    against the closed form in tests/test_gpu_qft33.py.)"""
    import synth
    from paper_2205_06973_gb300 import api
    n, g, x = synth.qft_basis(33)
    st = api.State(n, "c64")
    rows = []
    for m, k, tc, jit in (("beam", 6, True, False), ("beam", 6, 2, False), ("beam", 10, False, True),
                          ("beam", 12, False, True)):
        plan = api.Plan(g, n, m, k, dfs_trials=64 if k <= 6 else 16)
        stt = plan.stats("c64", tc=tc)
        cs = plan.specialise("c64", tc=tc) if jit else 0.0
        st.set_basis(x)
        ms = _timed(st, plan, tc=tc, jit=jit, reps=1)
        gbs = stt["passes"] * 2 * st.nbytes / (ms / 1e3) / 1e9
        rows.append({"method": m, "k": k, "tc": tc, "jit": jit, "passes": stt["passes"], "ms": round(ms, 1),
                     "GBs": round(gbs, 1), "frac": round(gbs / peak, 4), "compile_s": round(cs, 2)})
        plan.close()
    norm = st.probs()
    st.close()
    return {"workload": "33-qubit QFT (577 gates) on a seeded basis state, complex64 (64 GiB)", "rows": rows,
            "best": min(rows, key=lambda r: r["ms"]), "norm_after_last": norm}


def run_ours(a):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import synth
    from paper_2205_06973_gb300 import api

    n, gates = synth.layered_28q(n=a.n)
    # the end-to-end loop's pinned host buffers and device states, allocated
    # once at start (as a service allocates its staging buffers and states),
    # before the autotuner's many allocations
    S = max(2, a.e2e_states)
    if not a.no_e2e:
        host_in, host_out = pinned_buffers(n, S)
        e2e_states = [api.State(n, "c64", stream=torch.cuda.Stream()) for _ in range(S)]
    st = api.State(n, "c64", tile=a.tile)
    if a.k:
        choice = {"method": a.method, "k": a.k, "tc": int(a.tc), "tile": a.tile, "jit": bool(a.jit),
                  "regbits": a.regbits, "trials": []}
    else:
        from paper_2205_06973_gb300 import autotune
        choice = autotune.tune_state(f"layered{n}", n, gates, "c64", state=st, use_cache=False)
    k, tc, method = choice["k"], int(choice["tc"]), choice["method"]   # tc: 0, 1 dense parts, 2 paired
    jit = bool(choice.get("jit"))
    regbits = int(choice.get("regbits") or 0)
    if choice.get("tile"):
        st = api.State(n, "c64", tile=choice["tile"])
    from paper_2205_06973_gb300.autotune import BEAM_WIDTH
    plan = api.Plan(gates, n, method, k, dfs_trials=BEAM_WIDTH if method == "beam" else 16)
    stats = plan.stats("c64", choice.get("tile", 0), tc=tc, regbits=regbits)
    if jit:
        plan.specialise("c64", choice.get("tile", 0), tc=tc, regbits=regbits)
    passes = stats["passes"]
    bytes_per_pass = 2 * st.nbytes
    bytes_per_step = passes * bytes_per_pass

    for _ in range(max(a.warmup, 3)):
        st.apply(plan, tc=tc, jit=jit, regbits=regbits)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st.stream)
    for _ in range(a.steps):
        st.apply(plan, tc=tc, jit=jit, regbits=regbits)
    e1.record(st.stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / a.steps
    ms = max_over_ranks(ws, ms, dev)
    value = ws * bytes_per_step / (ms / 1e3) / 1e9
    norm = st.probs()

    # the step launches only the part kernel, back to back on the state's stream
    launch_ms = ms / passes
    peak, peak_kind = peaks()
    achieved = bytes_per_pass / (launch_ms / 1e3) / 1e9
    kernel = (("k_dense6_pair" if tc == 2 else "k_dense6") if (tc and stats["dense"] * 2 >= passes)
              else ("hisv_part" if jit else "k_part"))
    wkey = (f"layered{n}_{method}_k{k}_c64_{('tc2' if tc == 2 else 'tc') if tc else 't' + str(choice.get('tile') or 'auto')}"
            f"{'_jit' if jit else ''}{'_r' + str(regbits) if regbits else ''}")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "traffic": traffic_from_profile(kernel, wkey), "kernel": kernel,
                "algorithmic_bytes_per_launch": bytes_per_pass, "launch_ms": round(launch_ms, 4)}

    e2e = None
    if not a.no_e2e:
        e2e = e2e_loop(n, plan, tc, jit, regbits, choice.get("tile", 0) or 0, S, host_in, host_out, ws, dev,
                       bytes_per_step, states=e2e_states)
        e2e["host_buffers"] = "pinned, allocated at process start"
        e2e["device_states"] = "allocated at process start"
        for x in e2e_states:
            x.close()
        del host_in, host_out, e2e_states
        if ws == 1 and not a.no_e2e_child:
            # the same loop in a fresh process that loads the tuned plan, as a
            # service does after tuning (the autotuner caches its choice)
            fresh = e2e_child(n, method, k, tc, jit, regbits, choice.get("tile", 0) or 0, S)
            if "value" in fresh:
                fresh["in_process_after_autotune"] = {"value": e2e["value"], "ms_per_step": e2e["ms_per_step"]}
                e2e = fresh
            else:
                e2e["fresh_process"] = fresh

    compare = None
    if not a.no_compare:
        st.apply(plan, gatewise=True)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(st.stream)
        st.apply(plan, gatewise=True)
        g1.record(st.stream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1)
        compare = {"gate_by_gate_ms_per_step": round(gms, 3), "gate_passes": len(gates),
                   "gate_by_gate_GBs": round(len(gates) * bytes_per_pass / (gms / 1e3) / 1e9, 1),
                   "speedup_vs_gate_by_gate": round(gms / ms, 3)}

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu:
        pog, P = plan.export()
        cpu = cpu_baseline_oracle(n, gates, pog, P, max_parts=64, budget_s=20.0)
        cpu["sample"] += f" ({method} k={k} plan)"

    grid = c128 = alu = ml = q33 = None
    if rank == 0 and not a.no_grid:
        alu = alu_peaks()
        grid = grid_section(n, gates, st, peak, alu["fp32"])
        c128 = c128_section(n, gates, peak, alu["fp64"])
        alu = {k: round(v / 1e12, 3) for k, v in alu.items()}
        ml = multilevel_section(peak)
        q33 = qft33_section(peak)

    batch = serving = None
    if rank == 0 and not a.no_batch:
        batch = batch_section(a.batch_circuits)
    if rank == 0 and not a.no_serving:
        # the child gets the device to itself: return the blocks this process
        # cached for the sections above (the 64 GiB QFT state and others)
        import gc
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        serving = serving_child(a.serving_window)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws, "steps": a.steps,
                "warmup": max(a.warmup, 3), "ms_per_step": round(ms, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_TC if tc else DTYPE_FP32, "data": "synthetic",
                "config": {"workload": workload_text(n, len(gates)), "n_qubits": n,
                           "gates": len(gates), "method": method,
                           "k": k, "tensor_core_dense_parts": stats["dense"], "passes": passes,
                           "specialised_kernels": jit, "tile": choice.get("tile") or "default",
                           "register_bits": regbits or "default",
                           "phases": stats["phases"], "ops": stats["ops"],
                           "autotune_trials": choice.get("trials", []),
                           "state_bytes": st.nbytes, "parallelism": f"replicas x{ws}",
                           "l2": "state (2 GiB) larger than L2 (129 MB); no flush needed"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": passes * a.steps, "compare": compare, "norm": norm,
                "grid": grid, "c128": c128, "alu_peak_tflops": alu, "multilevel": ml, "qft33": q33,
                "batch": batch, "serving": serving}
        print(json.dumps(line), flush=True)
    st.close()
    plan.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(a):
    """The oracle timed on the host cores: each step is one part pass of the
    same plan in the oracle's Algorithm 1 mode (complex128)."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import synth
    from oracle import partition as opart
    from oracle import sim
    import numpy as np
    n, gates = synth.layered_28q(n=a.n)
    # k = 10 unless given: the oracle's Algorithm 1 pays per outer assignment,
    # so a k = 6 pass takes ~21 s on 16 Arm cores and a k = 10 pass ~3.3 s;
    # the metric (bytes of one whole-state part pass per second) is the same
    k = a.k or 10
    method = a.method if a.method in ("nat", "dfs", "dagp") else "dagp"
    pog = np.asarray(opart.partition(gates, n, method, k, seed=0), dtype=np.uint32)
    P = int(pog.max()) + 1
    parts = [[g for g, s in zip(gates, pog == p) if s] for p in range(P)]
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    step = 0

    def one():
        nonlocal psi, step
        sub = parts[step % P]
        psi = sim.run_alg1(n, sub, [0] * len(sub), 1, psi)
        step += 1

    for _ in range(a.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        one()
    dt = (time.perf_counter() - t0) / a.steps
    bytes_per_pass = 2 * 16 * (1 << n)
    value = bytes_per_pass / dt / 1e9
    cpu = {"value": round(value, 3), "unit": UNIT, "cores": sim.num_threads(), "kind": "oracle",
           "sample": f"one part pass per step ({a.steps} steps) of the {method} k={k} plan, "
                     "Algorithm 1 mode, complex128"}
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128 (fp64 arithmetic)", "data": "synthetic",
            "config": {"workload": workload_text(n, len(gates)).replace(
                           "complex64 state", "complex128 state (the oracle's type)"),
                       "n_qubits": n, "method": a.method, "k": k, "passes": P,
                       "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": cpu,
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _oracle_timing():
    """One measurement series of the oracle (complex128, OpenMP threads as
    set by OMP_NUM_THREADS): gate by gate and Algorithm 1 on the 14-qubit
    plain layered circuit (whole), the 28-qubit layered circuit (a prefix of
    gates / parts, scaled to the whole) and a sample of the 4096-circuit batch."""
    import numpy as np
    import synth
    from oracle import partition as pt
    from oracle import sim
    threads = sim.num_threads()

    def rec(**kw):
        kw["threads"] = threads
        kw["kind"] = "oracle"
        print(json.dumps(kw), flush=True)

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    n, g = synth.plain_layered_14q()
    rec(workload="plain layered 14q, 840 gates, complex128", mode="gate by gate",
        s=round(timed(lambda: sim.run(n, g)), 4), scaled="none")
    pog = pt.partition(g, n, "dagp", 8)
    P = max(pog) + 1
    rec(workload="plain layered 14q, 840 gates, complex128", mode=f"Algorithm 1, dagP k=8 ({P} parts)",
        s=round(timed(lambda: sim.run_alg1(n, g, pog, P)), 4), scaled="none")
    n, g = synth.layered_28q()
    psi = sim.basis(n)
    G0 = 8
    dt = timed(lambda: sim.run(n, g[:G0], psi))
    rec(workload="layered 28q, 2520 gates, complex128", mode="gate by gate", s=round(dt * len(g) / G0, 2),
        scaled=f"first {G0} gates took {dt:.2f} s, scaled by {len(g)}/{G0}")
    pog = np.asarray(pt.partition(g, n, "dagp", 10))
    P = int(pog.max()) + 1
    P0 = 1
    sub = [x for x, p in zip(g, pog) if p < P0]
    dt = timed(lambda: sim.run_alg1(n, sub, [int(p) for p in pog if p < P0], P0, psi))
    rec(workload="layered 28q, 2520 gates, complex128", mode=f"Algorithm 1, dagP k=10 ({P} parts)",
        s=round(dt * P / P0, 2), scaled=f"first {P0} parts took {dt:.2f} s, scaled by {P}/{P0}")
    circs = synth.batch_circuits(16)
    dt = timed(lambda: [sim.run(c[0], c[1]) for c in circs])
    rec(workload="4096 parameterised circuits, 10-20 qubits, complex128", mode="gate by gate",
        circuits_per_s=round(len(circs) / dt, 2), scaled=f"{len(circs)} circuits took {dt:.2f} s")
    plans = [pt.partition(c[1], c[0], "dfs", 9) for c in circs]
    dt = timed(lambda: [sim.run_alg1(c[0], c[1], p, max(p) + 1) for c, p in zip(circs, plans)])
    rec(workload="4096 parameterised circuits, 10-20 qubits, complex128", mode="Algorithm 1, DFS k=9",
        circuits_per_s=round(len(circs) / dt, 2), scaled=f"{len(circs)} circuits took {dt:.2f} s")


def oracle_report():
    """The oracle timing series single-threaded and on all host cores (each
    in a child process, since OpenMP reads its thread count at start)."""
    for threads in ("1", str(os.cpu_count() or 1)):
        env = dict(os.environ, OMP_NUM_THREADS=threads, HISV_ORACLE_TIMING="1")
        subprocess.run([sys.executable, os.path.abspath(__file__), "--impl", "reference"], env=env, check=True)


def partition_quality():
    """Part counts of the Nat, DFS, dagP and beam (width 16) builders against the exact
    optimum (SV_PART_EXACT; the comparison Sec. V-A makes with an ILP): 54
    small random layered circuits (6-8 qubits, depth 2-4, both gate sets, k
    3-5) and small instances of the benchmark families (QFT, layered,
    parameterised). One JSON line; host library only."""
    import synth
    from paper_2205_06973_gb300 import api

    def count(g, n, m, k):
        p = api.Plan(g, n, m, k)
        c = p.export()[1]
        p.close()
        return c

    def rows(cases):
        out = []
        for name, n, g, k in cases:
            t0 = time.perf_counter()
            opt = count(g, n, "exact", k)
            r = {"case": name, "gates": len(g), "k": k, "exact": opt, "exact_s": round(time.perf_counter() - t0, 3)}
            for m in ("nat", "dfs", "dagp", "beam"):
                r[m] = count(g, n, m, k)
            out.append(r)
        return out

    def summary(rs):
        s = {}
        for m in ("nat", "dfs", "dagp", "beam"):
            ex = [r[m] - r["exact"] for r in rs]
            s[m] = {"optimal": sum(e == 0 for e in ex), "of": len(rs),
                    "mean_excess_parts": round(sum(ex) / len(ex), 3), "max_excess_parts": max(ex),
                    "mean_ratio": round(sum(r[m] / r["exact"] for r in rs) / len(rs), 3)}
        return s

    rand = []
    for n in (6, 7, 8):
        for d in (2, 3, 4):
            for two_q in (("CX",), ("CX", "CZ")):
                for k in (3, 4, 5):
                    seed = 1000 * n + 100 * d + 10 * len(two_q) + k
                    rand.append((f"layered{n}d{d}{'cxcz' if len(two_q) > 1 else 'cx'}k{k}", n,
                                 synth.layered(n, d, seed=seed, two_q=two_q), k))
    fam = []
    for n, k in ((6, 3), (8, 4), (10, 5), (10, 4)):
        fam.append((f"qft{n}k{k}", n, synth.qft(n), k))
    for n, d, k in ((8, 5, 4), (10, 5, 5), (10, 6, 5), (10, 6, 6)):
        fam.append((f"layered{n}d{d}k{k}", n, synth.layered(n, d, seed=5), k))
    for n, d, k in ((8, 3, 4), (10, 3, 5), (10, 4, 5), (10, 4, 6)):
        fam.append((f"param{n}d{d}k{k}", n, synth.param(n, d, seed=4), k))
    r1, r2 = rows(rand), rows(fam)
    print(json.dumps({"partition_quality": {"random_small": summary(r1), "families": summary(r2),
                                            "family_cases": r2}}))
    print(json.dumps({"exchange_plans": exchange_report()}))


def exchange_report():
    """Exchanges of the distributed state (Sec. III-D) planned from each
    builder's first-level partition under L_m = l = n - p on 2^p ranks, for
    the 28-qubit layered circuit and the 33-qubit QFT: parts, all-to-all
    exchanges and qubits moved (host only)."""
    import synth
    from paper_2205_06973_gb300 import api
    from paper_2205_06973_gb300 import distributed as D
    rows = []
    n33, g33, _ = synth.qft_basis(33)
    for name, (n, g) in (("layered28", synth.layered_28q()), ("qft33", (n33, g33))):
        for p in (1, 2, 3):
            for m in ("nat", "dfs", "dagp", "beam"):
                pl = api.Plan(g, n, m, n - p)
                pog, P = pl.export()
                pl.close()
                qs = [set() for _ in range(P)]
                for i, x in enumerate(pog):
                    qs[x] |= set(g[i][1])
                ex, moved = D.count_exchanges([sorted(q) for q in qs], n, p)
                rows.append({"circuit": name, "ranks": 1 << p, "method": m, "parts": P, "exchanges": ex,
                             "qubits_moved": moved})
    return rows


def main():
    if os.environ.get("HISV_ORACLE_TIMING"):
        _oracle_timing()
        return
    a = parse()
    if a.partition_quality:
        partition_quality()
    elif a.serving_full:
        serving_full(a.serving_jit_large)
    elif a.serving_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"serving": serving_section(a.serving_window)}), flush=True)
    elif a.impl == "reference" and a.oracle_report:
        oracle_report()
    elif a.impl == "reference":
        run_reference(a)
    elif a.e2e_only:
        run_e2e_only(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
