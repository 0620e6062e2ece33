"""ctypes binding of ``libhisvsim.so`` (the C ABI in include/hisvsim.h).

Argument marshalling only: every step of the simulation runs in the native
library's CUDA kernels. Importing this module fails loudly when the library
has not been built; there is no Python or CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhisvsim.so")

SV_OK, SV_ERR_ARG, SV_ERR_OOM, SV_ERR_CUDA, SV_ERR_PARTITION, SV_ERR_TIMEOUT, SV_ERR_BUSY, SV_ERR_INTERNAL = range(8)
SV_C64, SV_C128, SV_C128DF = 0, 1, 2
PRECISIONS = {"c64": SV_C64, "c128": SV_C128, "c128df": SV_C128DF}
SV_PART_NONE, SV_PART_NAT, SV_PART_DFS, SV_PART_DAGP, SV_PART_EXACT, SV_PART_BEAM = 0, 1, 2, 3, 4, 5
METHODS = {"none": SV_PART_NONE, "nat": SV_PART_NAT, "dfs": SV_PART_DFS, "dagp": SV_PART_DAGP,
           "exact": SV_PART_EXACT, "beam": SV_PART_BEAM}
SV_FLAG_GATEWISE = 0x1
SV_FLAG_SYNC = 0x2
SV_FLAG_TC_DENSE = 0x4
SV_FLAG_SPECIALISE = 0x8
SV_FLAG_TC_PAIRS = 0x10


def tc_flags(tc):
    """Tensor-core flags for tc: False/0 none, True/1 dense parts, 2 dense
    parts with two per pass where they fit one tile."""
    if not tc:
        return 0
    return SV_FLAG_TC_DENSE | (SV_FLAG_TC_PAIRS if tc == 2 else 0)


def SV_FLAG_REGBITS(r):
    return (int(r) & 0xF) << 8


SV_NOALLOC_MAX_BLOCKS = 4096

GATE_KINDS = ("H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "P", "CX", "CZ", "CP", "SWAP")
KIND = {name: i for i, name in enumerate(GATE_KINDS)}


class sv_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint16), ("arity", ctypes.c_uint16),
                ("q", ctypes.c_uint32 * 3), ("theta", ctypes.c_double)]


assert ctypes.sizeof(sv_gate) == 24


class SvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the native library first "
        "(python -c 'import __graft_entry__ as g; g.build()' or python paper_2205_06973_gb300/build.py)")

lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_u32p = ctypes.POINTER(ctypes.c_uint32)
_SIGS = {
    "sv_create": ([ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_destroy": ([_vp], ctypes.c_int),
    "sv_attach": ([ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_set_basis": ([_vp, ctypes.c_uint64], ctypes.c_int),
    "sv_upload": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "sv_copy_state": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "sv_download": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "sv_batch_hold_last_item": ([_vp, ctypes.c_int], ctypes.c_int),
    "sv_qasm_parse": ([ctypes.c_char_p, _vp, _vp, _vp], ctypes.c_int),
    "sv_free_gates": ([_vp], None),
    "sv_export_c128": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "sv_device_ptr": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "sv_sync": ([_vp], ctypes.c_int),
    "sv_set_tile": ([_vp, ctypes.c_int], ctypes.c_int),
    "sv_plan_build": ([_vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                       ctypes.c_int, ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_plan_export": ([_vp, _vp, ctypes.c_size_t, _u32p], ctypes.c_int),
    "sv_plan_build_ml": ([_vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_plan_export_inner": ([_vp, _vp, ctypes.c_size_t, _u32p], ctypes.c_int),
    "sv_plan_stats": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, _u32p, _u32p, _u32p, _u32p], ctypes.c_int),
    "sv_plan_destroy": ([_vp], ctypes.c_int),
    "sv_plan_flops": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "sv_plan_specialise": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_int,
                            ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "sv_plan_source": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_char_p,
                        ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "sv_apply_parts": ([_vp, _vp, ctypes.c_uint32], ctypes.c_int),
    "sv_measure_probs": ([_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "sv_measure_summary": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "sv_batch_prepare": ([_vp], ctypes.c_int),
    "sv_alu_probe": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "sv_probs_noalloc": ([_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp], ctypes.c_int),
    "sv_batch_create": ([ctypes.c_uint32, _vp, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_batch_set_plan": ([_vp, ctypes.c_uint32, _vp], ctypes.c_int),
    "sv_batch_config": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "sv_batch_run": ([_vp, ctypes.c_uint32], ctypes.c_int),
    "sv_batch_reset": ([_vp], ctypes.c_int),
    "sv_batch_probs": ([_vp, _vp, _vp], ctypes.c_int),
    "sv_batch_state": ([_vp, ctypes.c_uint32, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "sv_batch_copy_state": ([_vp, ctypes.c_uint32, _vp, ctypes.c_size_t], ctypes.c_int),
    "sv_batch_info": ([_vp, ctypes.POINTER(ctypes.c_uint64), _u32p, _u32p], ctypes.c_int),
    "sv_batch_sync": ([_vp], ctypes.c_int),
    "sv_batch_set_dense": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "sv_batch_dense_info": ([_vp, _u32p, _u32p, _u32p], ctypes.c_int),
    "sv_batch_destroy": ([_vp], ctypes.c_int),
    "sv_last_error": ([], ctypes.c_char_p),
    "sv_version": ([], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def check(status: int):
    if status != SV_OK:
        raise SvError(status, lib.sv_last_error().decode())


def encode_gates(gates):
    """(name, qubits, theta) tuples -> ctypes array of sv_gate."""
    arr = (sv_gate * max(1, len(gates)))()
    for i, (name, qs, th) in enumerate(gates):
        g = arr[i]
        g.kind = KIND[name]
        g.arity = len(qs)
        for j, q in enumerate(qs):
            g.q[j] = q
        g.theta = th
    return arr
