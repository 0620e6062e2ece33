"""Parity at the benchmark's full size against the CPU oracle: the 28-qubit
random layered circuit (depth 60, 2520 gates) from |0...0>, computed once
per session by the oracle gate by gate in complex128 (psi_out = U_G ... U_1
psi_in, Sec. II-B; a few minutes on the host cores), then compared amplitude
by amplitude with every plan the state autotuner may pick for the benchmark
(tensor-core dense parts and gate-list parts) and with the configured
builders of Sec. IV-B (Nat / DFS / dagP) at k in {8, 10, 12}, each applied by
the library through the C ABI in the launch configuration bench.py times.

Bars (complex64 state): max-abs <= 1e-5, relative L2 error <= 1e-4,
fidelity |<ref|out>|^2 / (|ref|^2 |out|^2) >= 0.99999, and the norm within
1e-4 of one (the FP32 gate-list paths have no unitarity rescale; their norm
drifts by ~1e-6 per pass)."""
import numpy as np
import pytest
import torch

import synth
from oracle import sim
from tests.gpu_util import native

pytestmark = pytest.mark.gpu

MAX_ABS = 1e-5
REL_L2 = 1e-4
FIDELITY = 0.99999
NORM = 1e-4


@pytest.fixture(scope="module")
def layered28():
    n, g = synth.layered_28q()
    assert n == 28 and len(g) == 2520
    ref = sim.run(n, g)                       # complex128, gate by gate (oracle)
    assert abs(np.linalg.norm(ref) - 1.0) <= 1e-12
    ref_d = torch.from_numpy(ref).to("cuda")
    del ref
    return n, g, ref_d


def _compare(ref, out, chunk=1 << 24):
    """max |out - ref|, ||out - ref|| / ||ref||, the fidelity and ||out||,
    accumulated in FP64 over chunks of the two device vectors."""
    mx, d2, r2, o2 = 0.0, 0.0, 0.0, 0.0
    ip = torch.zeros((), dtype=torch.complex128, device=ref.device)
    for s in range(0, ref.numel(), chunk):
        r = ref[s:s + chunk]
        o = out[s:s + chunk].to(torch.complex128)
        d = o - r
        mx = max(mx, float(d.abs().max()))
        d2 += float((d.real ** 2 + d.imag ** 2).sum())
        r2 += float((r.real ** 2 + r.imag ** 2).sum())
        o2 += float((o.real ** 2 + o.imag ** 2).sum())
        ip += torch.vdot(r, o)
    fid = float(ip.abs() ** 2) / (r2 * o2)
    return mx, (d2 / r2) ** 0.5, fid, o2 ** 0.5


def _check(api, n, g, ref, method, k, tc=False, gatewise=False, dfs_trials=16, jit=False, regbits=0, tile=0):
    plan = api.Plan(g, n, method, k, dfs_trials=dfs_trials)
    st = api.State(n, "c64", tile=tile)
    st.apply(plan, sync=True, tc=tc, gatewise=gatewise, jit=jit, regbits=regbits)
    stats = plan.stats("c64", tile, tc=tc, regbits=regbits)
    mx, rel, fid, nrm = _compare(ref, st.amplitudes())
    st.close()
    plan.close()
    tag = (f"{method} k={k} tc={tc} jit={jit} tile={tile} regbits={regbits} gatewise={gatewise} "
           f"passes={stats['passes']} dense={stats['dense']}")
    assert mx <= MAX_ABS, f"{tag}: max-abs {mx:.3e}"
    assert rel <= REL_L2, f"{tag}: rel-L2 {rel:.3e}"
    assert fid >= FIDELITY, f"{tag}: fidelity {fid}"
    assert abs(nrm - 1.0) <= NORM, f"{tag}: norm {nrm}"
    return stats


def test_benchmark_plans_match_oracle(layered28):
    """Every candidate of the state autotuner against the oracle (the
    benchmark times the fastest of them: on GB300 the beam builder's k = 9
    plan on the specialised kernels, 79 passes)."""
    _, api = native()
    from paper_2205_06973_gb300.autotune import BEAM_WIDTH, STATE_CANDIDATES
    n, g, ref = layered28
    for cand in STATE_CANDIDATES:
        method, k, tc, tile, jit = cand[:5]
        regbits = cand[5] if len(cand) > 5 else 0
        stats = _check(api, n, g, ref, method, k, tc=tc, dfs_trials=BEAM_WIDTH if method == "beam" else 16,
                       jit=jit, regbits=regbits, tile=tile)
        if tc and k <= 6:
            assert stats["dense"] == stats["passes"]


@pytest.mark.parametrize("method,k", [("dagp", 8), ("dagp", 10), ("dagp", 12), ("nat", 10), ("dfs", 10)])
def test_paper_builders_match_oracle(layered28, method, k):
    """The paper's three builders at the configured limits, on the gate-list
    interpreter kernel and on the plan's specialised kernels."""
    _, api = native()
    n, g, ref = layered28
    _check(api, n, g, ref, method, k)
    _check(api, n, g, ref, method, k, jit=True)


@pytest.mark.parametrize("method,k", [("nat", 8), ("nat", 12), ("dfs", 8), ("dfs", 12)])
def test_builder_grid_matches_oracle(layered28, method, k):
    """The rest of the builder x k grid that bench.py times (Nat and DFS at
    k = 8 and 12), on both gate-list kernels."""
    _, api = native()
    n, g, ref = layered28
    _check(api, n, g, ref, method, k)
    _check(api, n, g, ref, method, k, jit=True)


@pytest.mark.parametrize("method", ["nat", "dfs", "dagp"])
def test_k12_on_its_own_tile_matches_oracle(layered28, method):
    """k = 12 parts on a 2^12 tile (the part's own qubits only, so a part
    without qubit 0 gathers runs of one amplitude), specialised kernels."""
    _, api = native()
    n, g, ref = layered28
    _check(api, n, g, ref, method, 12, jit=True, tile=12)


@pytest.mark.parametrize("method,k", [("dagp", 10), ("beam", 10), ("beam", 12)])
def test_multilevel_plans_match_oracle(layered28, method, k):
    """Two-level plans (Sec. IV-B): the first-level parts re-partitioned by a
    second builder under k2 = 5, whose parts are the register phases of the
    specialised kernels; the plans bench.py times beside one level."""
    _, api = native()
    n, g, ref = layered28
    for inner in (("dagp", 5), ("beam", 5)):
        plan = api.Plan(g, n, method, k, inner=inner)
        st = api.State(n, "c64")
        st.apply(plan, sync=True, jit=True)
        mx, rel, fid, nrm = _compare(ref, st.amplitudes())
        st.close()
        plan.close()
        tag = f"{method} k={k} inner={inner}"
        assert mx <= MAX_ABS, f"{tag}: max-abs {mx:.3e}"
        assert rel <= REL_L2, f"{tag}: rel-L2 {rel:.3e}"
        assert fid >= FIDELITY, f"{tag}: fidelity {fid}"
        assert abs(nrm - 1.0) <= NORM, f"{tag}: norm {nrm}"


def test_gate_by_gate_matches_oracle(layered28):
    _, api = native()
    n, g, ref = layered28
    _check(api, n, g, ref, "dagp", 10, gatewise=True)


def test_complex128_paths_match_oracle(layered28):
    """The 28-qubit circuit in complex128, the paper's precision, on the FP64
    interpreter kernel and on the plan's specialised kernels in FP64 and in
    double-float arithmetic (SV_C128DF): max-abs <= 1e-12 against the oracle."""
    _, api = native()
    n, g, ref = layered28
    # every row of the benchmark's complex128 section
    cases = (("dagp", 10, "c128", False), ("dagp", 10, "c128", True), ("beam", 10, "c128", False),
             ("beam", 10, "c128", True), ("beam", 10, "c128df", True), ("beam", 8, "c128df", True),
             ("dagp", 10, "c128df", True))
    for method, k, precision, jit in cases:
        plan = api.Plan(g, n, method, k, dfs_trials=16)
        st = api.State(n, precision)
        st.apply(plan, sync=True, jit=jit)
        out = st.amplitudes() if precision == "c128" else st.export_c128()
        mx = float(max((out[s:s + (1 << 24)] - ref[s:s + (1 << 24)]).abs().max() for s in range(0, 1 << n, 1 << 24)))
        del out
        st.close()
        plan.close()
        assert mx <= 1e-12, (method, k, precision, jit, mx)
