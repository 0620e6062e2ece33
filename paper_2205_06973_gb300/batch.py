"""Batched persistent launch over many small circuits (sv_batch_* of the C ABI).

All states live in one device buffer that the library allocates; ``Batch``
wraps the handle, keeps the plans alive and returns per-circuit
probabilities as views of one concatenated device tensor.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import os

import numpy as np
import torch

from . import _native as N
from .api import Plan


class Batch:
    def __init__(self, circuits, method="dfs", k=9, warps_per_cta=0, tiles_per_item=0, stream=None,
                 plans=None, dense_min_qubits=0, dense_tiles_per_item=0, dense_group_tiles=0,
                 dense_method="beam", dense_beam_width=4):
        """circuits: list of (n_qubits, gates); or plans: list of built Plan
        objects (the batch then owns them). dense_min_qubits > 0: circuits of
        at least max(dense_min_qubits, 13) qubits are planned with parts of at
        most 6 qubits and run on the batched tensor-core kernel (one fused
        64x64 unitary per part); the others keep k and the gate-list kernel.
        dense_tiles_per_item / dense_group_tiles: work-item size and the size
        of the L2-resident circuit groups of the dense work order, in 64 KiB
        tiles (0 = defaults 2 and 1024). dense_method / dense_beam_width: the
        part builder of the dense circuits (the beam builder halves the
        passes of the parameterised ladder circuits against DFS)."""
        if plans is not None:
            circuits = [(p.n, None) for p in plans]
        self.n = len(circuits)
        self.nq = np.array([c[0] for c in circuits], dtype=np.int32)
        self.offsets = np.concatenate([[0], np.cumsum(1 << self.nq.astype(np.int64))])
        self.total = int(self.offsets[-1])
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = ctypes.c_void_p()
        N.check(N.lib.sv_batch_create(self.n, self.nq.ctypes.data, ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.byref(h)))
        self.h = h
        if plans is None:   # the partitioners run in C++ with the GIL released: plan in parallel
            with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
                dmin = max(dense_min_qubits, 13) if dense_min_qubits else 0

                def plan(c):
                    if dmin and c[0] >= dmin:
                        return Plan(c[1], c[0], dense_method, 6, dfs_trials=dense_beam_width)
                    return Plan(c[1], c[0], method, min(k, c[0]))
                plans = list(ex.map(plan, circuits))
        self.plans = plans
        for i, p in enumerate(self.plans):
            N.check(N.lib.sv_batch_set_plan(self.h, i, p.h))
        if warps_per_cta or tiles_per_item:
            N.check(N.lib.sv_batch_config(self.h, warps_per_cta, tiles_per_item))
        if dense_min_qubits:
            N.check(N.lib.sv_batch_set_dense(self.h, dense_min_qubits, dense_tiles_per_item, dense_group_tiles))

    @classmethod
    def from_plans(cls, items, stream=None, warps_per_cta=0, tiles_per_item=0, dense_min_qubits=0):
        """items: list of (n_qubits, Plan). dense_min_qubits as for the
        constructor; the plans of those circuits must have parts of at most
        6 qubits to run on the batched tensor-core kernel."""
        return cls(None, plans=[p for _, p in items], stream=stream, warps_per_cta=warps_per_cta,
                   tiles_per_item=tiles_per_item, dense_min_qubits=dense_min_qubits)

    def configure(self, warps_per_cta=0, tiles_per_item=0):
        N.check(N.lib.sv_batch_config(self.h, warps_per_cta, tiles_per_item))

    def run(self, sync=False):
        N.check(N.lib.sv_batch_run(self.h, N.SV_FLAG_SYNC if sync else 0))

    def prepare(self):
        """Build the device program and capture the graph without launching."""
        N.check(N.lib.sv_batch_prepare(self.h))

    def reset(self):
        N.check(N.lib.sv_batch_reset(self.h))

    def sync(self):
        N.check(N.lib.sv_batch_sync(self.h))

    def probs(self, out=None, norms=True):
        """Probabilities of all states (one float32 device tensor, concatenated)
        and the per-circuit norms (numpy, FP64 accumulation) if requested."""
        if out is None:
            out = torch.empty(self.total, dtype=torch.float32, device="cuda")
        nrm = np.zeros(self.n, dtype=np.float64) if norms else None
        N.check(N.lib.sv_batch_probs(self.h, ctypes.c_void_p(out.data_ptr()),
                                     nrm.ctypes.data if norms else None))
        return out, nrm

    def state_host(self, i):
        """Circuit i's amplitudes copied to host memory (synchronises)."""
        host = torch.empty(1 << int(self.nq[i]), dtype=torch.complex64)
        N.check(N.lib.sv_batch_copy_state(self.h, i, ctypes.c_void_p(host.data_ptr()), host.numel() * 8))
        return host

    def info(self):
        t, it, pa = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
        N.check(N.lib.sv_batch_info(self.h, ctypes.byref(t), ctypes.byref(it), ctypes.byref(pa)))
        dc, di, dp = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        N.check(N.lib.sv_batch_dense_info(self.h, ctypes.byref(dc), ctypes.byref(di), ctypes.byref(dp)))
        return {"amplitudes": t.value, "items": it.value, "parts": pa.value,
                "dense_circuits": dc.value, "dense_items": di.value, "dense_passes": dp.value}

    def close(self):
        if getattr(self, "h", None):
            N.lib.sv_batch_destroy(self.h)
            self.h = None
        for p in getattr(self, "plans", []):
            p.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
