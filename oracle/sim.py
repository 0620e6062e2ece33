"""ctypes front-end of the C oracle ``sv_oracle.c`` (test infrastructure).

Builds ``liborc.so`` next to the source with gcc on first use (or from
``__graft_entry__.build()``) and exposes complex128 numpy entry points:

* ``run(n, gates, state)``      - gate-by-gate simulation (Sec. II-B / III-A)
* ``run_alg1(n, gates, part_of_gate, n_parts, state, order_mode)``
                                 - Algorithm 1 Gather-Execute-Scatter
* ``run_alg1_nested(n, gates, outer, inner, state)``
                                 - Algorithm 1 with nested parts (multi-level)
* ``probs(state)``               - |a_x|^2 and their sum

Gates are ``(name, qubits, theta)`` tuples as produced by ``synth``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

# this file's own gate numbering; must match the enum in sv_oracle.c
_CODES = {"H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "T": 5, "RX": 6, "RY": 7,
          "RZ": 8, "P": 9, "CX": 10, "CZ": 11, "CP": 12, "SWAP": 13}

OGATE = np.dtype([("kind", np.int32), ("nq", np.int32), ("q", np.int32, (2,)),
                  ("theta", np.float64)])


def build(force: bool = False) -> str:
    """Compile liborc.so (gcc, OpenMP) if missing or older than the source."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_run.argtypes = [dp, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_run_alg1.argtypes = [dp, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int]
        lib.orc_run_alg1.restype = ctypes.c_int
        lib.orc_probs.argtypes = [dp, ctypes.c_int, dp]
        lib.orc_probs.restype = ctypes.c_double
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def encode(gates) -> np.ndarray:
    arr = np.zeros(len(gates), dtype=OGATE)
    for i, (name, qs, th) in enumerate(gates):
        arr[i]["kind"] = _CODES[name]
        arr[i]["nq"] = len(qs)
        for j, q in enumerate(qs):
            arr[i]["q"][j] = q
        arr[i]["theta"] = th
    return arr


def basis(n: int, x: int = 0) -> np.ndarray:
    s = np.zeros(1 << n, dtype=np.complex128)
    s[x] = 1.0
    return s


def _prep(n, state):
    if state is None:
        state = basis(n, 0)
    s = np.ascontiguousarray(state, dtype=np.complex128).copy()
    if s.shape != (1 << n,):
        raise ValueError("state must have 2^n entries")
    return s


def run(n: int, gates, state=None) -> np.ndarray:
    s = _prep(n, state)
    enc = encode(gates)
    rc = _load().orc_run(s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n,
                         enc.ctypes.data, len(enc))
    if rc:
        raise ValueError(f"oracle run failed ({rc})")
    return s


def run_alg1(n: int, gates, part_of_gate, n_parts: int, state=None, order_mode: int = 0):
    s = _prep(n, state)
    enc = encode(gates)
    pog = np.ascontiguousarray(part_of_gate, dtype=np.uint32)
    if len(pog) != len(enc):
        raise ValueError("part_of_gate length mismatch")
    rc = _load().orc_run_alg1(s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n,
                              enc.ctypes.data, len(enc), pog.ctypes.data, n_parts, order_mode)
    if rc:
        raise ValueError(f"oracle alg1 failed ({rc})")
    return s


def run_alg1_nested(n: int, gates, outer, inner, state=None):
    """Algorithm 1 with nested parts (the multi-level execution of Sec. IV-B):
    for every first-level part, in order, and every assignment of the qubits
    outside it, gather the part's inner state vector (local bit j = the j-th
    smallest qubit of the part), run Algorithm 1 of its second-level parts on
    that vector with the gates' qubits renamed to local bits, and scatter it
    back. outer / inner: first- and second-level part of every gate (inner
    numbered over the circuit, each part's inner parts contiguous)."""
    s = _prep(n, state)
    outer = [int(x) for x in outer]
    inner = [int(x) for x in inner]
    P = (max(outer) + 1) if outer else 0
    for p in range(P):
        ids = [g for g in range(len(gates)) if outer[g] == p]
        S = sorted({q for g in ids for q in gates[g][1]})
        O = [q for q in range(n) if q not in S]
        w = len(S)
        local = {q: j for j, q in enumerate(S)}
        sub = [(gates[g][0], tuple(local[q] for q in gates[g][1]), gates[g][2]) for g in ids]
        first = min(inner[g] for g in ids)
        sub_pog = [inner[g] - first for g in ids]
        n_sub = max(sub_pog) + 1
        y = np.arange(1 << w, dtype=np.int64)
        idx_in = np.zeros(1 << w, dtype=np.int64)
        for j, q in enumerate(S):
            idx_in |= ((y >> j) & 1) << q
        a = np.arange(1 << len(O), dtype=np.int64)
        idx_out = np.zeros(1 << len(O), dtype=np.int64)
        for j, q in enumerate(O):
            idx_out |= ((a >> j) & 1) << q
        for base in idx_out:
            x = base | idx_in
            s[x] = run_alg1(w, sub, sub_pog, n_sub, s[x])
    return s


def probs(state: np.ndarray):
    s = np.ascontiguousarray(state, dtype=np.complex128)
    n = int(np.log2(len(s)))
    p = np.empty(len(s), dtype=np.float64)
    tot = _load().orc_probs(s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n,
                            p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return p, tot


def num_threads() -> int:
    return _load().orc_num_threads()
