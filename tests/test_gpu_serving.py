"""Serving loop: continuous batching with admission by state bytes. Each
request's result is the same alone and in the mix (complex64 tolerance), the
gate-by-gate serving mode gives the same states, and the byte budget bounds
what is resident."""
import numpy as np
import pytest

import synth
from oracle import sim
from tests.gpu_util import native

pytestmark = pytest.mark.gpu


def _stream(count, seed=5, max_n=22):
    out = []
    arr = synth.serving_arrivals(count, duration_s=0.5, seed=seed)
    i = 0
    while len(out) < count:
        n, fam, g = synth.serving_request(i, seed=seed)
        i += 1
        if n > max_n:
            continue
        out.append((n, fam, g, arr[len(out)]))
    return out


def test_alone_equals_in_the_mix_and_oracle():
    native()
    from paper_2205_06973_gb300.serving import Request, Server
    stream = _stream(24)
    reqs = [Request(i, n, g, t, fam) for i, (n, fam, g, t) in enumerate(stream)]
    srv = Server(budget_bytes=64e6, small_n=18, keep_states=True, k_large=6)
    mix, stats = srv.run(reqs)
    assert stats["requests"] == len(reqs)
    for r in mix:
        assert abs(r.norm - 1.0) < 1e-4
    for j in (0, 5, 11, 17, 23):
        r = reqs[j]
        alone, _ = Server(budget_bytes=64e6, small_n=18, keep_states=True, k_large=6).run(
            [Request(0, r.n, r.gates, 0.0)])
        a = alone[0].state.numpy()
        m = mix[j].state.numpy()
        assert np.abs(a - m).max() <= 1e-6, j
        if r.n <= 16:
            ref = sim.run(r.n, r.gates)
            assert np.abs(m - ref).max() <= 1e-5, j


def test_gatewise_serving_matches():
    native()
    from paper_2205_06973_gb300.serving import Request, Server
    stream = _stream(8, seed=7, max_n=16)
    reqs = [Request(i, n, g, t) for i, (n, fam, g, t) in enumerate(stream)]
    a, _ = Server(small_n=18, keep_states=True).run(reqs)
    b, _ = Server(small_n=18, keep_states=True, mode="gatewise").run(reqs)
    for x, y in zip(a, b):
        assert np.abs(x.state.numpy() - y.state.numpy()).max() <= 1e-5


def test_budget_limits_residency():
    native()
    from paper_2205_06973_gb300.serving import Request, Server
    # four 20-qubit states of 8 MiB each with a 17 MiB budget: at most two resident
    g = synth.layered(20, 4, seed=1, two_q=("CX", "CZ"))
    reqs = [Request(i, 20, g, 0.0) for i in range(4)]
    res, stats = Server(budget_bytes=17 * 2 ** 20, small_n=18, k_large=6).run(reqs)
    starts = sorted(r.start for r in res)
    dones = sorted(r.done for r in res)
    # the third request can only start after one of the first two finished
    assert starts[2] >= dones[0] - 1e-6
    assert stats["requests"] == 4


def test_served_mix_fidelity():
    """Every result of a served mix (10-24 qubits, the three families) has
    fidelity >= 0.99999 against an FP64 reference: the CPU oracle for
    n <= 20, the closed form for the QFT family of any size (QFT of |0...0>),
    else the complex128 gate-list path (FP64, pinned to the oracle by the
    parity tests)."""
    import torch
    from oracle import closed_form as cf
    _, api = native()
    from paper_2205_06973_gb300.serving import Request, Server
    stream = _stream(32, seed=13, max_n=24)
    reqs = [Request(i, n, g, t, fam) for i, (n, fam, g, t) in enumerate(stream)]
    assert any(r.n > 20 for r in reqs) and any(r.family == "qft" and r.n > 20 for r in reqs)
    res, _ = Server(keep_states=True).run(reqs)
    for r, out in zip(reqs, res):
        psi = out.state.numpy().astype(np.complex128)
        if r.family == "qft":
            ref = cf.qft_state(sim.basis(r.n))
        elif r.n <= 20:
            ref = sim.run(r.n, r.gates)
        else:
            plan = api.Plan(r.gates, r.n, "dagp", 10)
            st = api.State(r.n, "c128")
            st.apply(plan, sync=True)
            ref = st.copy_to_host().numpy()
            st.close()
            plan.close()
        fid = abs(np.vdot(ref, psi)) ** 2
        assert fid >= 0.99999, (r.rid, r.n, r.family, fid)
        assert np.abs(psi - ref).max() <= 1e-5, (r.rid, r.n, r.family)


def test_large_requests_of_the_stream():
    """A seeded sample of the serving stream's requests of 25-28 qubits (the
    first four, seed 5), served together through admission and the large-
    request path: each state has fidelity >= 0.99999 and max-abs <= 1e-5
    against an FP64 reference (the closed form for the QFT family, the CPU
    oracle up to 26 qubits, else the complex128 gate-list path), and the
    device summary (norm, |a_0|^2, most likely state) matches the state."""
    import torch
    from oracle import closed_form as cf
    _, api = native()
    from paper_2205_06973_gb300.serving import Request, Server
    arr = synth.serving_arrivals(20000, 60.0, seed=5)
    reqs, i = [], 0
    while len(reqs) < 4:
        n, fam, g = synth.serving_request(i, seed=5)
        if 25 <= n <= 28:
            reqs.append(Request(len(reqs), n, g, arr[i] - arr[0] if reqs else 0.0, fam))
        i += 1
    srv = Server(budget_bytes=170e9, keep_states=True)
    res, stats = srv.run(reqs)
    srv.close()
    assert stats["requests"] == 4
    for r, out in zip(reqs, res):
        psi = out.state.numpy().astype(np.complex128)
        if r.family == "qft":
            ref = cf.qft_state(sim.basis(r.n))
        elif r.n <= 26:
            ref = sim.run(r.n, r.gates)
        else:
            plan = api.Plan(r.gates, r.n, "dagp", 10)
            st = api.State(r.n, "c128")
            st.apply(plan, sync=True)
            ref = st.copy_to_host().numpy()
            st.close()
            plan.close()
        fid = abs(np.vdot(ref, psi)) ** 2
        assert fid >= 0.99999, (r.rid, r.n, r.family, fid)
        assert np.abs(psi - ref).max() <= 1e-5, (r.rid, r.n, r.family)
        p = psi.real ** 2 + psi.imag ** 2
        assert abs(out.norm - p.sum()) <= 1e-6, r.rid
        assert abs(out.p0 - p[0]) <= 1e-9, r.rid
        assert abs(out.pmax - p.max()) <= 1e-9 and p[out.argmax] >= p.max() - 1e-9, r.rid
        del psi, ref, p
        torch.cuda.empty_cache()
