"""GPU parity of the dense tensor-core part path (SV_FLAG_TC_DENSE): parts of
at most 6 qubits applied as one fused 64x64 unitary in split BF16 with FP32
accumulation, against the CPU oracle (max-abs 1e-5, relative L2 1e-4)."""
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


@pytest.mark.parametrize("n", [12, 13, 14, 17])
def test_dense_layered(n):
    _, g = synth.layered_28q(n=n, depth=8)
    psi = random_state(n, 2 + n)
    ref = sim.run(n, g, psi)
    for method, k in (("nat", 6), ("dagp", 6), ("dagp", 4)):
        out = run_gpu(n, g, method=method, k=k, psi=psi, tc=True)
        assert max_abs(out, ref) <= 1e-5, (method, k)
        assert rel_l2(out, ref) <= 1e-4, (method, k)


def test_dense_high_qubits_and_all_kinds():
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
    out = run_gpu(n, g, method="dagp", k=6, psi=psi, tc=True)
    assert max_abs(out, ref) <= 1e-5
    assert rel_l2(out, ref) <= 1e-4


def test_dense_qft_closed_form():
    n = 18
    x = synth.SplitMix64(21).randint(1 << n)
    ref = cf.qft_basis_amplitude(n, x, np.arange(1 << n))
    out = run_gpu(n, synth.qft(n), method="dagp", k=6, basis=x, tc=True)
    assert max_abs(out, ref) <= 1e-5
    assert rel_l2(out, ref) <= 1e-4


def test_dense_stats_and_mixed_plan():
    _, api = native()
    n, g = synth.layered_28q(n=16, depth=10)
    plan = api.Plan(g, n, "dagp", 8)
    s = plan.stats("c64", tc=True)
    assert 0 < s["dense"] < s["passes"]          # parts of 7-8 qubits stay on the gate-list kernel
    ref = sim.run(n, g)
    out = run_gpu(n, g, method="dagp", k=8, tc=True)
    assert max_abs(out, ref) <= 1e-5


def test_dense_norm_and_fidelity_deep_circuit():
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
    out = run_gpu(n, g, method="dagp", k=6, psi=psi, tc=True)
    assert abs(float(np.vdot(out, out).real) - 1.0) <= 5e-6
    assert abs(np.vdot(ref, out)) ** 2 >= 0.99999
    assert max_abs(out, ref) <= 1e-5
