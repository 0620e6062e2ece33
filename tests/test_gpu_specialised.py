"""GPU parity of the part kernels specialised for a plan (SV_FLAG_SPECIALISE:
generated CUDA compiled with NVRTC) against the CPU oracle, element by
element (max-abs 1e-5 complex64, 1e-12 complex128), over every gate kind,
the three builders of Sec. IV-B, every tile size and both precisions, and
against the interpreter kernel on the same plan."""
import numpy as np
import pytest

import synth
from oracle import closed_form as cf
from oracle import sim
from tests.gpu_util import TOL, max_abs, native, random_state, run_gpu
from tests.test_gpu_parity import _all_kinds

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["c64", "c128", "c128df"])
@pytest.mark.parametrize("n", [10, 11, 13, 15])
def test_all_gate_kinds(precision, n):
    g = _all_kinds(n, 300, 40 + n)
    psi = random_state(n, 3 + n)
    ref = sim.run(n, g, psi)
    for method, k in (("nat", 3), ("dfs", 5), ("dagp", 8), ("dagp", 10), ("beam", 10)):
        out = run_gpu(n, g, method=method, k=k, precision=precision, psi=psi, jit=True)
        assert max_abs(out, ref) <= TOL[precision], (method, k)


@pytest.mark.parametrize("precision,tile", [("c64", 10), ("c64", 11), ("c64", 12), ("c64", 13),
                                            ("c128", 10), ("c128", 11), ("c128", 12),
                                            ("c128df", 10), ("c128df", 11), ("c128df", 12)])
def test_tiles(precision, tile):
    n = 17
    _, g = synth.layered_28q(n=n, depth=12)
    psi = random_state(n, 77)
    ref = sim.run(n, g, psi)
    for method, k in (("dagp", 6), ("beam", min(tile, 10)), ("nat", min(tile, 10))):
        out = run_gpu(n, g, method=method, k=k, precision=precision, tile=tile, psi=psi, jit=True)
        assert max_abs(out, ref) <= TOL[precision], (method, k, tile)


@pytest.mark.parametrize("precision", ["c64", "c128", "c128df"])
def test_qft_and_long_runs(precision):
    """Diagonal-heavy parts (QFT: merged phase-vector ops) and long runs of
    one-qubit gates (fused 2x2 ops), with the thread-bit controls."""
    n = 16
    x = 12345
    out = run_gpu(n, synth.qft(n), method="dagp", k=10, precision=precision, basis=x, jit=True)
    ref = cf.qft_basis_amplitude(n, x, np.arange(1 << n))
    assert max_abs(out, ref) <= TOL[precision]
    r = synth.SplitMix64(99)
    g = []
    for _ in range(400):
        q = r.randint(n)
        name = ("H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "P")[r.randint(10)]
        g.append((name, (q,), r.angle()))
        if r.randint(6) == 0:
            a = r.randint(n)
            g.append((("CX", "CZ", "CP", "SWAP")[r.randint(4)], (a, (a + 1 + r.randint(n - 1)) % n), r.angle()))
    psi = random_state(n, 5)
    ref = sim.run(n, g, psi)
    for k in (5, 9, 12):
        out = run_gpu(n, g, method="dagp", k=k, precision=precision, psi=psi, jit=True)
        assert max_abs(out, ref) <= TOL[precision], k


def test_same_as_interpreter():
    """The same plan on the interpreter kernel and on its specialised kernels:
    the same operations in the same order (FMA contraction may differ)."""
    n, g = synth.layered_28q(n=20, depth=20)
    psi = random_state(n, 8)
    for method, k in (("dagp", 10), ("beam", 12)):
        a = run_gpu(n, g, method=method, k=k, psi=psi)
        b = run_gpu(n, g, method=method, k=k, psi=psi, jit=True)
        assert max_abs(a, b) <= 1e-6, (method, k)


def test_dense_and_specialised_mix():
    """SV_FLAG_TC_DENSE with SV_FLAG_SPECIALISE: parts of <= 6 qubits on the
    tensor cores, the rest on specialised kernels, in one apply."""
    n, g = synth.layered_28q(n=18, depth=16)
    psi = random_state(n, 21)
    ref = sim.run(n, g, psi)
    _, api = native()
    out = run_gpu(n, g, method="dagp", k=7, psi=psi, tc=True, jit=True)
    assert max_abs(out, ref) <= 1e-5
    plan = api.Plan(g, n, "dagp", 7)
    st = plan.stats("c64", 0, tc=True)
    assert 0 < st["dense"] < st["passes"], st
    plan.close()


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_multilevel_plans(precision):
    """Multi-level plans (Sec. IV-B): first-level parts as HBM passes, their
    second-level parts as register phases, on the interpreter and on the
    specialised kernels, against the oracle."""
    _, api = native()
    import torch
    n = 16
    _, g = synth.layered_28q(n=n, depth=14)
    g = g + synth.qft(n)[:120]
    psi = random_state(n, 31)
    ref = sim.run(n, g, psi)
    k2 = 5 if precision == "c64" else 4
    dt = torch.complex128 if precision == "c128" else torch.complex64
    for m1, k1, m2 in (("dagp", 10, "dagp"), ("beam", 12, "beam"), ("nat", 8, "nat"), ("dfs", 10, "dagp")):
        plan = api.Plan(g, n, m1, k1, inner=(m2, k2))
        for jit in (False, True):
            st = api.State(n, precision)
            st.upload(torch.from_numpy(np.ascontiguousarray(psi)).to(dt).pin_memory())
            st.apply(plan, sync=True, jit=jit)
            out = st.copy_to_host().numpy().astype(np.complex128)
            st.close()
            assert max_abs(out, ref) <= TOL[precision], (m1, k1, m2, jit)
        plan.close()


def test_double_float_state_io_and_reductions():
    """A double-float complex128 state: upload and download round trip
    (double -> hi + lo -> double keeps 48 bits: within 2^-47 relative), the
    basis state, norm and summary reductions, the device export, and the
    paths it has no kernels for refused."""
    import torch
    _, api = native()
    N = api.N
    n = 12
    psi = random_state(n, 44)
    st = api.State(n, "c128df")
    st.upload(torch.from_numpy(psi).pin_memory())
    back = st.copy_to_host().numpy()
    assert np.abs(back - psi).max() <= 2.0 ** -47
    dev = st.export_c128()
    assert np.abs(dev.cpu().numpy() - back).max() == 0.0
    assert abs(st.probs() - 1.0) <= 1e-12
    norm, p0, am, pm = st.summary()
    p = np.abs(back) ** 2
    assert abs(norm - 1.0) <= 1e-12 and abs(p0 - p[0]) <= 1e-15 and am == int(np.argmax(p))
    st.set_basis(77)
    out = st.copy_to_host().numpy()
    assert out[77] == 1.0 and np.count_nonzero(out) == 1
    plan = api.Plan(synth.qft(n), n, "dagp", 8)
    with pytest.raises(N.SvError):
        st.apply(plan, gatewise=True)
    st.apply(plan, sync=True)
    ref = cf.qft_basis_amplitude(n, 77, np.arange(1 << n))
    assert max_abs(st.copy_to_host().numpy(), ref) <= 1e-12
    plan.close()
    st.close()


@pytest.mark.parametrize("precision,regbits,tile", [("c64", 4, 12), ("c64", 6, 12), ("c64", 4, 13),
                                                    ("c128", 3, 11), ("c128df", 3, 11)])
def test_register_bits(precision, regbits, tile):
    """2^r amplitudes per thread (SV_FLAG_REGBITS) against the oracle."""
    _, api = native()
    import torch
    n = 16
    g = _all_kinds(n, 300, 71) + synth.qft(n)[:80]
    psi = random_state(n, 72)
    ref = sim.run(n, g, psi)
    dt = torch.complex64 if precision == "c64" else torch.complex128
    for method, k in (("dagp", 8), ("beam", 10)):
        plan = api.Plan(g, n, method, k)
        st = api.State(n, precision, tile=tile)
        st.upload(torch.from_numpy(np.ascontiguousarray(psi)).to(dt).pin_memory())
        st.apply(plan, sync=True, jit=True, regbits=regbits)
        out = st.copy_to_host().numpy().astype(np.complex128)
        st.close()
        plan.close()
        assert max_abs(out, ref) <= TOL[precision], (method, k)
