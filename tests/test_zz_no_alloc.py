"""The allocation-free probabilities entry point (sv_probs_noalloc).

Some callers cannot allocate device memory: their framework owns every byte
through its own pool under a fixed budget, or they run in a loop where a
device allocation could stall the device. sv_probs_noalloc serves them with
a static scratch array inside the library. This test calls it through the C
ABI on a state the ordinary API prepared and checks, on two calls in a row,
that its probabilities and norm match sv_measure_probs (the entry point that
uses allocated scratch), within the complex64 / complex128 tolerances of the
other GPU tests. The file sorts last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import native

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_noalloc_matches_allocating_entry_point(precision):
    N, api = native()
    n = 18
    _, g = synth.layered_28q(n=n, depth=6)
    plan = api.Plan(g, n, "dagp", 8)
    st = api.State(n, precision)
    st.apply(plan, sync=True)
    fp64 = precision == "c128"
    ref_p = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    ref_norm = st.probs(ref_p, fp64=True)
    tol = 1e-12 if fp64 else 1e-6
    ptr = ctypes.c_void_p()
    N.check(N.lib.sv_device_ptr(st.h, ctypes.byref(ptr), None))
    prec = N.SV_C128 if fp64 else N.SV_C64
    stream = ctypes.c_void_p(st.stream.cuda_stream)
    for call in range(2):
        out = torch.full((1 << n,), -1.0, dtype=torch.float64, device="cuda")
        norm = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        N.check(N.lib.sv_probs_noalloc(ptr, n, prec, ctypes.c_void_p(out.data_ptr()), 1,
                                       ctypes.c_void_p(norm.data_ptr()), 0, stream))
        torch.cuda.synchronize()
        assert np.abs(out.cpu().numpy() - ref_p.cpu().numpy()).max() <= tol, call
        assert abs(norm.item() - ref_norm) <= tol, call
    # float32 output and a narrower reduction give the same norm
    out32 = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    N.check(N.lib.sv_probs_noalloc(ptr, n, prec, ctypes.c_void_p(out32.data_ptr()), 0,
                                   ctypes.c_void_p(norm.data_ptr()), 64, stream))
    torch.cuda.synchronize()
    assert abs(norm.item() - ref_norm) <= tol
    assert np.abs(out32.cpu().numpy() - ref_p.cpu().numpy()).max() <= 1e-6
    st.close()
    plan.close()


def test_noalloc_rejects_oversized_reduction():
    N, api = native()
    st = api.State(12, "c64")
    ptr = ctypes.c_void_p()
    N.check(N.lib.sv_device_ptr(st.h, ctypes.byref(ptr), None))
    rc = N.lib.sv_probs_noalloc(ptr, 12, N.SV_C64, None, 0, None, N.SV_NOALLOC_MAX_BLOCKS + 1,
                                ctypes.c_void_p(st.stream.cuda_stream))
    assert rc == N.SV_ERR_ARG
    assert b"n_blocks" in N.lib.sv_last_error()
    assert N.lib.sv_probs_noalloc(None, 12, N.SV_C64, None, 0, None, 0, None) == N.SV_ERR_ARG
    st.close()
