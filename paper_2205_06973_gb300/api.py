"""Thin Python front-end over the C ABI: ``Plan`` and ``State`` handles.

PyTorch provides the device memory (a uint8 tensor owns the amplitudes) and
the CUDA stream; every computation is a call into ``libhisvsim.so``.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N


class Plan:
    """sv_plan_build: DAG + partition (Sec. IV) of a circuit, host only."""

    def __init__(self, gates, n, method="dagp", k=10, seed=0, dfs_trials=16, inner=None):
        """inner = (method2, k2): multi-level partitioning (sv_plan_build_ml),
        every part re-partitioned with method2 under k2."""
        self.n = n
        self.G = len(gates)
        self.method = method
        self.k = k
        self.inner = inner
        self._arr = N.encode_gates(gates)
        h = ctypes.c_void_p()
        if inner is None:
            N.check(N.lib.sv_plan_build(ctypes.cast(self._arr, ctypes.c_void_p), self.G, n, N.METHODS[method],
                                        k, seed, dfs_trials, ctypes.byref(h)))
        else:
            N.check(N.lib.sv_plan_build_ml(ctypes.cast(self._arr, ctypes.c_void_p), self.G, n, N.METHODS[method],
                                           k, N.METHODS[inner[0]], inner[1], seed, dfs_trials, ctypes.byref(h)))
        self.h = h

    def export_inner(self):
        """Second-level part of every gate and their count (multi-level plans)."""
        import numpy as np
        inner = np.zeros(max(1, self.G), dtype=np.uint32)
        P = ctypes.c_uint32()
        N.check(N.lib.sv_plan_export_inner(self.h, inner.ctypes.data, self.G, ctypes.byref(P)))
        return inner[: self.G], P.value

    def export(self):
        import numpy as np
        pog = np.zeros(max(1, self.G), dtype=np.uint32)
        P = ctypes.c_uint32()
        N.check(N.lib.sv_plan_export(self.h, pog.ctypes.data, self.G, ctypes.byref(P)))
        return pog[: self.G], P.value

    def stats(self, precision="c64", tile=0, tc=False, regbits=0):
        a, b, c, d = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        N.check(N.lib.sv_plan_stats(self.h, N.PRECISIONS[precision], tile,
                                    N.tc_flags(tc) | N.SV_FLAG_REGBITS(regbits),
                                    ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
        return {"passes": a.value, "phases": b.value, "ops": c.value, "dense": d.value}

    def flops(self, precision="c64", tile=0, tc=False, gatewise=False):
        """(CUDA-core flops, tensor-core flops) of one apply (sv_plan_flops)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        flags = N.tc_flags(tc) | (N.SV_FLAG_GATEWISE if gatewise else 0)
        N.check(N.lib.sv_plan_flops(self.h, N.PRECISIONS[precision], tile, flags,
                                    ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def specialise(self, precision="c64", tile=0, tc=False, load=True, regbits=0):
        """Generate and compile the plan's specialised part kernels
        (SV_FLAG_SPECIALISE) now; load=False only compiles (no device).
        regbits: amplitudes per thread 2^regbits (0 = default). Returns the
        compile time in seconds."""
        s = ctypes.c_double()
        N.check(N.lib.sv_plan_specialise(self.h, N.PRECISIONS[precision], tile,
                                         N.tc_flags(tc) | N.SV_FLAG_REGBITS(regbits),
                                         1 if load else 0, ctypes.byref(s)))
        return s.value

    def source(self, part, precision="c64", tile=0, tc=False, regbits=0):
        """Generated CUDA source of gate-list part ``part``."""
        n = ctypes.c_size_t()
        args = (self.h, N.PRECISIONS[precision], tile,
                N.tc_flags(tc) | N.SV_FLAG_REGBITS(regbits), part)
        N.check(N.lib.sv_plan_source(*args, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value + 1)
        N.check(N.lib.sv_plan_source(*args, buf, n.value + 1, ctypes.byref(n)))
        return buf.value.decode()

    def close(self):
        if self.h:
            N.lib.sv_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """sv_create over a torch-owned device buffer on the current stream."""

    def __init__(self, n, precision="c64", device="cuda", stream=None, tile=0):
        """precision: "c64", "c128", or "c128df" (complex128 held as
        double-float pairs, computed on the FP32 pipes; see SV_C128DF)."""
        self.n = n
        self.precision = precision
        self.amp_bytes = 8 if precision == "c64" else 16
        self.nbytes = self.amp_bytes << n
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.buf.device)
        h = ctypes.c_void_p()
        N.check(N.lib.sv_create(n, N.PRECISIONS[precision],
                                ctypes.c_void_p(self.buf.data_ptr()), self.nbytes,
                                ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        if tile:
            N.check(N.lib.sv_set_tile(self.h, tile))

    @classmethod
    def over(cls, amps, n, precision="c64", stream=None, tile=0):
        """A state handle over an existing CUDA tensor of 2^n complex
        amplitudes (sv_attach: the contents are kept, the tensor stays owned
        by the caller)."""
        self = cls.__new__(cls)
        self.n = n
        self.precision = precision
        self.amp_bytes = 8 if precision == "c64" else 16
        self.nbytes = self.amp_bytes << n
        assert amps.is_cuda and amps.numel() * amps.element_size() == self.nbytes and amps.is_contiguous()
        self.buf = amps
        self.stream = stream if stream is not None else torch.cuda.current_stream(amps.device)
        h = ctypes.c_void_p()
        N.check(N.lib.sv_attach(n, N.PRECISIONS[precision],
                                ctypes.c_void_p(amps.data_ptr()), self.nbytes,
                                ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        if tile:
            N.check(N.lib.sv_set_tile(self.h, tile))
        return self

    # views of the amplitudes (no copy)
    def amplitudes(self):
        """The amplitudes as a complex tensor view (complex64 / complex128
        states; a double-float state gives a complex128 copy, export_c128)."""
        if self.precision == "c128df":
            return self.export_c128()
        dt = torch.complex128 if self.precision == "c128" else torch.complex64
        return self.buf.view(dt)

    def export_c128(self, out=None):
        """Complex128 device tensor of the amplitudes (sv_export_c128,
        stream-ordered on the state's stream)."""
        if out is None:
            out = torch.empty(1 << self.n, dtype=torch.complex128, device=self.buf.device)
        N.check(N.lib.sv_export_c128(self.h, ctypes.c_void_p(out.data_ptr()), out.numel() * 16))
        return out

    def set_tile(self, tile_qubits):
        """CTA tile of the part kernels for this state (sv_set_tile; 0 = default)."""
        N.check(N.lib.sv_set_tile(self.h, tile_qubits))

    def set_basis(self, x):
        N.check(N.lib.sv_set_basis(self.h, x))

    def upload(self, host_tensor):
        t = host_tensor.contiguous()
        assert t.numel() * t.element_size() == self.nbytes
        N.check(N.lib.sv_upload(self.h, ctypes.c_void_p(t.data_ptr()), self.nbytes))

    def copy_to_host(self, out=None):
        dt = torch.complex64 if self.precision == "c64" else torch.complex128
        if out is None:
            out = torch.empty(1 << self.n, dtype=dt)
        N.check(N.lib.sv_copy_state(self.h, ctypes.c_void_p(out.data_ptr()), self.nbytes))
        return out

    def download(self, out):
        """Stream-ordered copy into the host tensor ``out`` (pinned for an
        asynchronous copy); the data is there after ``sync()``."""
        N.check(N.lib.sv_download(self.h, ctypes.c_void_p(out.data_ptr()), self.nbytes))
        return out

    def apply(self, plan: Plan, gatewise=False, sync=False, tc=False, jit=False, regbits=0):
        flags = ((N.SV_FLAG_GATEWISE if gatewise else 0) | (N.SV_FLAG_SYNC if sync else 0)
                 | N.tc_flags(tc) | (N.SV_FLAG_SPECIALISE if jit else 0)
                 | N.SV_FLAG_REGBITS(regbits))
        N.check(N.lib.sv_apply_parts(self.h, plan.h, flags))

    def probs(self, out=None, fp64=False):
        norm = ctypes.c_double()
        ptr = ctypes.c_void_p(out.data_ptr()) if out is not None else None
        N.check(N.lib.sv_measure_probs(self.h, ptr, 1 if fp64 else 0, ctypes.byref(norm)))
        return norm.value

    def summary(self):
        """(norm, |a_0|^2, argmax_x |a_x|^2, max |a_x|^2) in FP64 without a
        probability vector (sv_measure_summary; synchronises)."""
        nrm, p0, pm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        am = ctypes.c_uint64()
        N.check(N.lib.sv_measure_summary(self.h, ctypes.byref(nrm), ctypes.byref(p0), ctypes.byref(am),
                                         ctypes.byref(pm)))
        return nrm.value, p0.value, am.value, pm.value

    def sync(self):
        N.check(N.lib.sv_sync(self.h))

    def close(self):
        if getattr(self, "h", None):
            N.lib.sv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
