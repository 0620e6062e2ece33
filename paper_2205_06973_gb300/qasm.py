"""OpenQASM 2.0 programs as gate lists (sv_qasm_parse of the C ABI).

    n, gates = qasm.loads(text)        # gates: [(name, qubits, theta), ...]
    n, gates = qasm.load(path)

The gate list feeds ``api.Plan`` like any other circuit. The conventions and
the exact decompositions of gates outside the library's set are stated at
sv_qasm_parse in include/hisvsim.h.
"""
from __future__ import annotations

import ctypes

from . import _native as N

_NAMES = {v: k for k, v in N.KIND.items()}


def loads(text: str):
    """Parse a program text; returns (n_qubits, gates)."""
    arr = ctypes.POINTER(N.sv_gate)()
    ng = ctypes.c_size_t()
    nq = ctypes.c_int()
    N.check(N.lib.sv_qasm_parse(text.encode(), ctypes.byref(arr), ctypes.byref(ng), ctypes.byref(nq)))
    try:
        gates = []
        for i in range(ng.value):
            g = arr[i]
            gates.append((_NAMES[g.kind], tuple(int(g.q[j]) for j in range(g.arity)), float(g.theta)))
    finally:
        N.lib.sv_free_gates(arr)
    return nq.value, gates


def load(path: str):
    with open(path) as f:
        return loads(f.read())
