"""The part kernels generated for a plan (SV_FLAG_SPECIALISE), built for the
host: the CUDA source of every part, as sv_plan_source returns it, is
compiled with g++ against tests/jit_host/host_prelude.h (plain C++ meanings
of the run-time prelude's helpers, one std::thread per CUDA thread of one
CTA, a std::barrier for __syncthreads) and run pass after pass on a small
state; the result must match the oracle (Sec. II-B: psi_out = U_G ... U_1
psi_in; Algorithm 1 applies it part by part) within the tolerances of the
GPU tests. This checks the generator's layouts, register phases and
straight-line gate arithmetic without a GPU; the device build of the same
source is checked against the oracle by the GPU tests."""
import os
import re
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import synth
from oracle import sim
from tests.test_gpu_parity import _all_kinds

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2205_06973_gb300", "csrc")
HOST = os.path.join(ROOT, "tests", "jit_host")
TOL = {"c64": 1e-5, "c128": 1e-12, "c128df": 1e-12}

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")

MAIN = r"""
#include <cstdio>
#include <thread>
#include <vector>
typedef void (*part_fn)(hisv::C *, unsigned long long);
static part_fn parts[] = {%(table)s};
int main(int argc, char **argv) {
    using namespace hisv;
    const int n = %(n)d, t = %(t)d, nt = %(nt)d;
    const size_t N = size_t(1) << n;
    std::vector<double> in(2 * N);
    FILE *f = std::fopen(argv[1], "rb");
    if (!f || std::fread(in.data(), sizeof(double), 2 * N, f) != 2 * N) return 2;
    std::fclose(f);
    std::vector<C> sv(N);
    for (size_t i = 0; i < N; i++) {
#if HISV_DF
        const float rh = (float)in[2 * i], ih = (float)in[2 * i + 1];
        sv[i].x = df(rh, (float)(in[2 * i] - (double)rh));
        sv[i].y = df(ih, (float)(in[2 * i + 1] - (double)ih));
#else
        sv[i].x = (Real)in[2 * i];
        sv[i].y = (Real)in[2 * i + 1];
#endif
    }
    for (part_fn p : parts) {
        std::barrier<> bar(nt);
        hisv_host_barrier = &bar;
        std::vector<std::thread> th;
        for (int tid = 0; tid < nt; tid++)
            th.emplace_back([&, tid] {
                threadIdx.x = tid;
                p(sv.data(), 1ull << (n - t));
            });
        for (auto &x : th) x.join();
    }
    for (size_t i = 0; i < N; i++) {
#if HISV_DF
        in[2 * i] = (double)sv[i].x.hi + (double)sv[i].x.lo;
        in[2 * i + 1] = (double)sv[i].y.hi + (double)sv[i].y.lo;
#else
        in[2 * i] = sv[i].x;
        in[2 * i + 1] = sv[i].y;
#endif
    }
    f = std::fopen(argv[2], "wb");
    if (!f || std::fwrite(in.data(), sizeof(double), 2 * N, f) != 2 * N) return 3;
    std::fclose(f);
    return 0;
}
"""


def _api():
    from paper_2205_06973_gb300 import build
    build.build()
    from paper_2205_06973_gb300 import api
    return api


def run_host(n, gates, method, k, precision="c64", tile=0, regbits=0, psi=None):
    """Apply the plan's generated kernels, built for the host, to psi."""
    api = _api()
    plan = api.Plan(gates, n, method, k)
    P = plan.stats(precision, tile, regbits=regbits)["passes"]
    srcs = [plan.source(i, precision, tile, regbits=regbits) for i in range(P)]
    plan.close()
    m = re.search(r"__launch_bounds__\((\d+),", srcs[0])
    nt = int(m.group(1))
    t = int(re.search(r"buf1 = buf0 \+ (\d+);", srcs[0]).group(1)).bit_length() - 1
    R = t - (nt.bit_length() - 1)
    body = "#include \"host_prelude.h\"\n" + "".join(srcs)
    body += MAIN % {"table": ", ".join(f"hisv_part_{i}" for i in range(P)), "n": n, "t": t, "nt": nt}
    fp64 = precision != "c64"
    with tempfile.TemporaryDirectory() as d:
        cpp, exe = os.path.join(d, "parts.cpp"), os.path.join(d, "parts")
        with open(cpp, "w") as f:
            f.write(body)
        subprocess.run(["g++", "-std=c++20", "-O1", "-pthread", "-w", f"-DHISV_R={R}",
                        f"-DHISV_FP64={int(fp64)}", f"-DHISV_DF={int(precision == 'c128df')}",
                        "-I", HOST, "-I", CSRC, cpp, "-o", exe], check=True)
        v = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128))
        v.view(np.float64).tofile(os.path.join(d, "in.bin"))
        subprocess.run([exe, os.path.join(d, "in.bin"), os.path.join(d, "out.bin")], check=True)
        out = np.fromfile(os.path.join(d, "out.bin"), dtype=np.float64).view(np.complex128)
    return out


def _psi(n, seed):
    a = synth.random_amplitudes(n, seed)
    v = a[:, 0] + 1j * a[:, 1]
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("precision", ["c64", "c128", "c128df"])
def test_all_gate_kinds_host(precision):
    n = 12
    g = _all_kinds(n, 200, 41)
    psi = _psi(n, 5)
    ref = sim.run(n, g, psi)
    for method, k in (("dagp", 8), ("beam", 10)):
        out = run_host(n, g, method, k, precision, psi=psi)
        assert np.abs(out - ref).max() <= TOL[precision], (method, k)


@pytest.mark.parametrize("tile,regbits", [(10, 0), (11, 0), (12, 4), (13, 0), (12, 6)])
def test_layered_tiles_host(tile, regbits):
    n, g = synth.layered_28q(n=14, depth=8)
    psi = _psi(n, 9)
    ref = sim.run(n, g, psi)
    for method, k in (("beam", min(tile, 10)), ("nat", 6)):
        out = run_host(n, g, method, k, "c64", tile=tile, regbits=regbits, psi=psi)
        assert np.abs(out - ref).max() <= TOL["c64"], (method, k, tile, regbits)


def test_qft_and_one_qubit_runs_host():
    n = 13
    r = synth.SplitMix64(99)
    g = list(synth.qft(n))
    for _ in range(150):
        q = r.randint(n)
        name = ("H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "P")[r.randint(10)]
        g.append((name, (q,), r.angle()))
        if r.randint(6) == 0:
            a = r.randint(n)
            g.append((("CX", "CZ", "CP", "SWAP")[r.randint(4)], (a, (a + 1 + r.randint(n - 1)) % n), r.angle()))
    psi = _psi(n, 4)
    ref = sim.run(n, g, psi)
    for k in (5, 9, 12):
        out = run_host(n, g, "dagp", k, "c64", psi=psi)
        assert np.abs(out - ref).max() <= TOL["c64"], k
