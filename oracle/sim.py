"""ctypes front-end of the C oracle ``sv_oracle.c`` (test infrastructure).

Builds ``liborc.so`` next to the source with gcc on first use (or from
``__graft_entry__.build()``) and exposes complex128 numpy entry points:

* ``run(n, gates, state)``      - gate-by-gate simulation (Sec. II-B / III-A)
* ``run_alg1(n, gates, part_of_gate, n_parts, state, order_mode)``
                                 - Algorithm 1 Gather-Execute-Scatter
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


def probs(state: np.ndarray):
    s = np.ascontiguousarray(state, dtype=np.complex128)
    n = int(np.log2(len(s)))
    p = np.empty(len(s), dtype=np.float64)
    tot = _load().orc_probs(s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n,
                            p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return p, tot


def num_threads() -> int:
    return _load().orc_num_threads()
