"""Host checks of the plan-specialised part kernels (SV_FLAG_SPECIALISE):
the generated CUDA source compiles with NVRTC for sm_103a (no device needed)
for every op kind and both precisions, and describes the part it came
from."""
import re

import pytest

import synth
from tests.test_gpu_parity import _all_kinds


def _api():
    from paper_2205_06973_gb300 import build
    build.build()
    from paper_2205_06973_gb300 import _native as N
    from paper_2205_06973_gb300 import api
    return N, api


@pytest.mark.parametrize("precision", ["c64", "c128", "c128df"])
def test_generated_source_compiles(precision):
    N, api = _api()
    n = 13
    g = _all_kinds(n, 300, 53) + synth.qft(n)
    plan = api.Plan(g, n, "dagp", 8)
    st = plan.stats(precision)
    src = "".join(plan.source(i, precision) for i in range(st["passes"]))
    # every op kind of the interpreter appears in the generated code
    h = ("op_h2<", "op_rys2<") if precision == "c64" else ("op_h<", "op_rys<")
    for name in h + ("op_u2s<", "op_rxs<", "op_x<", "op_y<", "op_p<", "op_cx<", "op_cz<",
                 "op_cp<", "op_cxt<", "tmul(", "cmul_in("):
        assert name in src, name
    assert len(re.findall(r'extern "C" __global__', src)) == st["passes"]
    secs = plan.specialise(precision, load=False)
    assert secs > 0.0
    plan.close()


def test_source_layout_and_errors():
    N, api = _api()
    n, g = synth.layered_28q(n=16, depth=6)
    plan = api.Plan(g, n, "nat", 10)
    src = plan.source(0, "c64", tile=12)
    assert "__launch_bounds__(128, 3)" in src          # 2^(12-5) threads, 3 CTAs of 64 KiB per SM
    assert "buf0 + 4096" in src
    with pytest.raises(N.SvError):
        plan.source(0, "c64", tile=9)                  # below the smallest tile
    with pytest.raises(N.SvError):
        plan.source(10 ** 6, "c64")                    # no such part
    plan.close()


def test_register_bits_variants():
    """SV_FLAG_REGBITS: 2^r amplitudes per thread in the specialised kernels
    (r = 4 and 6 for complex64, 3 for complex128): the programs compile with
    NVRTC, the CTA has 2^(t - r) threads, and out-of-range choices fail."""
    N, api = _api()
    n, g = synth.layered_28q(n=16, depth=6)
    plan = api.Plan(g, n, "beam", 9)
    for prec, r, t in (("c64", 4, 12), ("c64", 6, 12), ("c64", 4, 13), ("c128", 3, 11)):
        src = plan.source(0, prec, tile=t, regbits=r)
        assert f"__launch_bounds__({1 << (t - r)}," in src, (prec, r, t)
        assert plan.specialise(prec, tile=t, load=False, regbits=r) > 0.0
    assert plan.stats("c64", 12, regbits=4)["phases"] >= plan.stats("c64", 12)["phases"]
    with pytest.raises(N.SvError):
        plan.stats("c64", 10, regbits=6)            # 2^4 threads: less than a warp
    plan.close()
