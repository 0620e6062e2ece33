"""GPU parity of the dense tensor-core part path (SV_FLAG_TC_DENSE): parts of
at most 6 qubits applied as one fused 64x64 unitary in split BF16 with FP32
accumulation, against the CPU oracle (max-abs 1e-5, relative L2 1e-4); with
SV_FLAG_TC_PAIRS (tc=2) two consecutive such parts share one pass over a
13-qubit tile (the second level of Sec. IV-B's multi-level partitioning)."""
import numpy as np
import pytest

import synth
from oracle import closed_form as cf
from oracle import sim
from tests.gpu_util import max_abs, native, random_state, run_gpu

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def test_dense_single_tile_identity_like():
    """13 qubits = one CTA tile; a part of one H then H again is the identity."""
    n = 13
    g = [("H", (0,), 0.0), ("H", (0,), 0.0)]
    psi = random_state(n, 1)
    out = run_gpu(n, g, method="nat", k=6, psi=psi, tc=True)
    assert max_abs(out, psi) <= 1e-5


@pytest.mark.parametrize("tc", [True, 2])
@pytest.mark.parametrize("n", [12, 13, 14, 17])
def test_dense_layered(n, tc):
    _, g = synth.layered_28q(n=n, depth=8)
    psi = random_state(n, 2 + n)
    ref = sim.run(n, g, psi)
    for method, k in (("nat", 6), ("dagp", 6), ("dagp", 4), ("beam", 6)):
        out = run_gpu(n, g, method=method, k=k, psi=psi, tc=tc)
        assert max_abs(out, ref) <= 1e-5, (method, k)
        assert rel_l2(out, ref) <= 1e-4, (method, k)


@pytest.mark.parametrize("tc", [True, 2])
def test_dense_high_qubits_and_all_kinds(tc):
    n = 16
    r = synth.SplitMix64(9)
    g = []
    for _ in range(200):
        name = synth.GATE_NAMES[r.randint(len(synth.GATE_NAMES))]
        if name in synth.TWO_QUBIT:
            a = 8 + r.randint(8)
            b = 8 + (a - 8 + 1 + r.randint(7)) % 8
            g.append((name, (a, b), r.angle()))
        else:
            g.append((name, (8 + r.randint(8),), r.angle()))
    psi = random_state(n, 3)
    ref = sim.run(n, g, psi)
    out = run_gpu(n, g, method="dagp", k=6, psi=psi, tc=tc)
    assert max_abs(out, ref) <= 1e-5
    assert rel_l2(out, ref) <= 1e-4


@pytest.mark.parametrize("tc", [True, 2])
def test_dense_qft_closed_form(tc):
    n = 18
    x = synth.SplitMix64(21).randint(1 << n)
    ref = cf.qft_basis_amplitude(n, x, np.arange(1 << n))
    for method in ("dagp", "beam"):
        out = run_gpu(n, synth.qft(n), method=method, k=6, basis=x, tc=tc)
        assert max_abs(out, ref) <= 1e-5, method
        assert rel_l2(out, ref) <= 1e-4, method


def test_dense_stats_and_mixed_plan():
    _, api = native()
    n, g = synth.layered_28q(n=16, depth=10)
    plan = api.Plan(g, n, "dagp", 8)
    s = plan.stats("c64", tc=True)
    assert 0 < s["dense"] < s["passes"]          # parts of 7-8 qubits stay on the gate-list kernel
    ref = sim.run(n, g)
    out = run_gpu(n, g, method="dagp", k=8, tc=True)
    assert max_abs(out, ref) <= 1e-5


@pytest.mark.parametrize("tc", [True, 2])
def test_dense_norm_and_fidelity_deep_circuit(tc):
    """Many dense passes: the norm stays at its input value (the passes rescale
    to it, the exact evolution being unitary) and the fidelity against the
    FP64 oracle stays >= 0.99999."""
    _, api = native()
    n = 16
    _, g = synth.layered_28q(n=n, depth=60)
    plan = api.Plan(g, n, "dagp", 6)
    assert plan.stats("c64", tc=True)["dense"] >= 60
    plan.close()
    psi = random_state(n, 31)
    ref = sim.run(n, g, psi)
    out = run_gpu(n, g, method="dagp", k=6, psi=psi, tc=tc)
    assert abs(float(np.vdot(out, out).real) - 1.0) <= 5e-6
    assert abs(np.vdot(ref, out)) ** 2 >= 0.99999
    assert max_abs(out, ref) <= 1e-5


def test_pairs_halve_the_passes_and_mix():
    """SV_FLAG_TC_PAIRS: consecutive dense parts share a pass (about half the
    passes of the dense plan), in one apply with single dense passes and
    gate-list parts (Nat k = 7 leaves its 7-qubit parts on the gate-list
    kernel), on the interpreter and on the specialised kernels."""
    _, api = native()
    n, g = synth.layered_28q(n=18, depth=20)
    plan = api.Plan(g, n, "beam", 6, dfs_trials=16)
    one, two = plan.stats("c64", tc=True), plan.stats("c64", tc=2)
    assert two["passes"] <= one["passes"] // 2 + 4 and two["dense"] == two["passes"]
    assert plan.flops("c64", tc=2)[1] == plan.flops("c64", tc=True)[1]
    plan.close()
    psi = random_state(n, 12)
    ref = sim.run(n, g, psi)
    plan = api.Plan(g, n, "nat", 7)
    mix = plan.stats("c64", tc=2)
    assert 0 < mix["dense"] < mix["passes"] < plan.stats("c64", tc=True)["passes"]
    plan.close()
    for method, k, jit in (("nat", 7, False), ("nat", 7, True), ("beam", 6, False)):
        out = run_gpu(n, g, method=method, k=k, psi=psi, tc=2, jit=jit)
        assert max_abs(out, ref) <= 1e-5, (method, k, jit)
        assert rel_l2(out, ref) <= 1e-4, (method, k, jit)
