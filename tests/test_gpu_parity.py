"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element, at sizes the oracle finishes in seconds. Tolerances:
max-abs 1e-5 for the complex64 state, 1e-12 for complex128."""
import numpy as np
import pytest
import torch

import synth
from oracle import closed_form as cf
from oracle import sim
from tests.gpu_util import TOL, max_abs, native, random_state, run_gpu

pytestmark = pytest.mark.gpu


def _all_kinds(n, G, seed):
    r = synth.SplitMix64(seed)
    gates = []
    for _ in range(G):
        name = synth.GATE_NAMES[r.randint(len(synth.GATE_NAMES))]
        if name in synth.TWO_QUBIT:
            a = r.randint(n)
            b = (a + 1 + r.randint(n - 1)) % n
            gates.append((name, (a, b), r.angle()))
        else:
            gates.append((name, (r.randint(n),), r.angle()))
    return gates


def test_cuda_available():
    assert torch.cuda.is_available()


@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_plain_layered_14q_gatewise(precision):
    """14 qubits, 840 gates, one pass per gate, all 16384 amplitudes."""
    n, g = synth.plain_layered_14q()
    ref = sim.run(n, g)
    out = run_gpu(n, g, gatewise=True, precision=precision)
    assert max_abs(out, ref) <= TOL[precision]


@pytest.mark.parametrize("precision", ["c128", "c64"])
@pytest.mark.parametrize("method", ["nat", "dfs", "dagp"])
def test_plain_layered_14q_parts(precision, method):
    n, g = synth.plain_layered_14q()
    ref = sim.run(n, g)
    for k in (4, 8, 10):
        out = run_gpu(n, g, method=method, k=k, precision=precision)
        assert max_abs(out, ref) <= TOL[precision], (method, k)


@pytest.mark.parametrize("precision", ["c64", "c128"])
@pytest.mark.parametrize("n", [10, 11, 13, 15])
def test_all_gate_kinds_parts(precision, n):
    g = _all_kinds(n, 300, 40 + n)
    psi = random_state(n, 3 + n)
    ref = sim.run(n, g, psi)
    for method, k in (("nat", 3), ("dfs", 5), ("dagp", 8), ("dagp", 10)):
        out = run_gpu(n, g, method=method, k=k, precision=precision, psi=psi)
        assert max_abs(out, ref) <= TOL[precision], (method, k)


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_all_gate_kinds_gatewise(precision):
    n = 12
    g = _all_kinds(n, 200, 9)
    psi = random_state(n, 10)
    ref = sim.run(n, g, psi)
    out = run_gpu(n, g, gatewise=True, precision=precision, psi=psi)
    assert max_abs(out, ref) <= TOL[precision]


@pytest.mark.parametrize("tile", [10, 11, 12, 13])
def test_tiles_c64(tile):
    n = 17
    n_, g = synth.layered_28q(n=n, depth=12)
    psi = random_state(n, 77)
    ref = sim.run(n, g, psi)
    for k in (6, min(tile, 10)):
        out = run_gpu(n, g, method="dagp", k=k, precision="c64", tile=tile, psi=psi)
        assert max_abs(out, ref) <= TOL["c64"], k


@pytest.mark.parametrize("tile", [10, 11, 12])
def test_tiles_c128(tile):
    n = 16
    _, g = synth.layered_28q(n=n, depth=10)
    psi = random_state(n, 78)
    ref = sim.run(n, g, psi)
    out = run_gpu(n, g, method="dfs", k=min(tile, 9), precision="c128", tile=tile, psi=psi)
    assert max_abs(out, ref) <= TOL["c128"]


@pytest.mark.parametrize("method", ["nat", "dfs", "dagp"])
@pytest.mark.parametrize("k", [8, 10, 12])
def test_layered_20q_parts(method, k):
    """The 28-qubit layered workload's recipe at 20 qubits (depth 20)."""
    n, g = synth.layered_28q(n=20, depth=20)
    ref = sim.run(n, g)
    for precision in ("c64", "c128"):
        if precision == "c128" and k > 12:
            continue
        out = run_gpu(n, g, method=method, k=k, precision=precision)
        assert max_abs(out, ref) <= TOL[precision]


@pytest.mark.parametrize("k,tc", [(6, True), (8, False), (10, False)])
def test_beam_plans(k, tc):
    """Plans of the beam part builder (fewer passes than dagP on the
    benchmark circuits) on the tensor-core and gate-list paths: the
    layered recipe at 20 qubits and a QFT of a basis state at 16 qubits
    against the oracle and the closed form."""
    n, g = synth.layered_28q(n=20, depth=20)
    ref = sim.run(n, g)
    out = run_gpu(n, g, method="beam", k=k, precision="c64", tc=tc)
    assert max_abs(out, ref) <= TOL["c64"]
    if not tc:
        out = run_gpu(n, g, method="beam", k=k, precision="c128")
        assert max_abs(out, ref) <= TOL["c128"]
    x = synth.SplitMix64(19).randint(1 << 16)
    ref = cf.qft_basis_amplitude(16, x, np.arange(1 << 16))
    out = run_gpu(16, synth.qft(16), method="beam", k=k, precision="c64", basis=x, tc=tc)
    assert max_abs(out, ref) <= TOL["c64"]


@pytest.mark.parametrize("n", [10, 14, 18])
def test_qft_basis_closed_form(n):
    x = synth.SplitMix64(3 + n).randint(1 << n)
    g = synth.qft(n)
    ref = cf.qft_basis_amplitude(n, x, np.arange(1 << n))
    for method, k in (("nat", 6), ("dagp", 10)):
        out = run_gpu(n, g, method=method, k=k, precision="c64", basis=x)
        assert max_abs(out, ref) <= TOL["c64"]
        out = run_gpu(n, g, method=method, k=k, precision="c128", basis=x)
        assert max_abs(out, ref) <= TOL["c128"]


def test_param_family():
    for i in range(3):
        n, g = synth.batch_circuit(i)
        if n > 16:
            continue
        ref = sim.run(n, g)
        out = run_gpu(n, g, method="dagp", k=10, precision="c64")
        assert max_abs(out, ref) <= TOL["c64"]


def test_small_n_runs_gatewise():
    n = 6
    g = _all_kinds(n, 80, 5)
    ref = sim.run(n, g)
    out = run_gpu(n, g, method="dagp", k=4, precision="c128")
    assert max_abs(out, ref) <= TOL["c128"]


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_probs_and_norm(precision):
    N_, api = native()
    n = 16
    _, g = synth.layered_28q(n=n, depth=6)
    ref = sim.run(n, g)
    plan = api.Plan(g, n, "dagp", 8)
    st = api.State(n, precision)
    st.apply(plan)
    for fp64 in (False, True):
        out = torch.empty(1 << n, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
        norm = st.probs(out, fp64=fp64)
        p = out.cpu().numpy()
        assert abs(norm - 1.0) < (1e-5 if precision == "c64" else 1e-12)
        # float32 output rounds each probability to 24 bits
        tol = 1e-13 if (precision == "c128" and fp64) else 1e-6
        assert np.abs(p - np.abs(ref) ** 2).max() < tol
    assert abs(st.probs() - 1.0) < 1e-5
    st.close()
    plan.close()


def test_empty_circuit_and_basis():
    out = run_gpu(12, [], method="dagp", k=8, basis=37)
    ref = np.zeros(1 << 12)
    ref[37] = 1
    assert max_abs(out, ref) == 0.0


def _one_qubit_runs(n, G, seed):
    """Long runs of one-qubit gates of every kind on few qubits, between
    sparse two-qubit gates: the planner fuses each run into one op (a phase
    when the product is diagonal, else a general 2x2 matrix)."""
    r = synth.SplitMix64(seed)
    one = [x for x in synth.GATE_NAMES if x not in synth.TWO_QUBIT]
    gates = []
    for _ in range(G):
        if r.randint(8) == 0:
            a = r.randint(n)
            b = (a + 1 + r.randint(n - 1)) % n
            gates.append((synth.TWO_QUBIT[r.randint(len(synth.TWO_QUBIT))], (a, b), r.angle()))
        else:
            q = r.randint(4)   # few qubits: long runs on each
            gates.append((one[r.randint(len(one))], (q,), r.angle()))
    # runs whose product is diagonal or the identity
    gates += [("H", (5,), 0.0), ("Z", (5,), 0.0), ("H", (5,), 0.0), ("X", (6,), 0.0), ("X", (6,), 0.0),
              ("RZ", (7,), 0.3), ("T", (7,), 0.0), ("S", (7,), 0.0)]
    return gates


@pytest.mark.parametrize("precision", ["c64", "c128"])
@pytest.mark.parametrize("method", ["nat", "dagp"])
def test_fused_one_qubit_runs(precision, method):
    n = 12
    g = _one_qubit_runs(n, 400, 77)
    psi = random_state(n, 78)
    ref = sim.run(n, g, psi)
    out = run_gpu(n, g, method=method, k=8, psi=psi, precision=precision)
    assert max_abs(out, ref) <= TOL[precision]


def test_download_stream_ordered():
    """sv_download queues the copy on the state's stream; after sv_sync the
    host buffer holds the state, also with a part pass queued before it."""
    _, api = native()
    n = 14
    psi = random_state(n, 91)
    g = synth.plain_layered_14q()[1][:60]
    ref = sim.run(n, g, psi)
    plan = api.Plan(g, n, "dagp", 8)
    st = api.State(n, "c64", stream=torch.cuda.Stream())
    st.upload(torch.from_numpy(psi).to(torch.complex64).pin_memory())
    st.apply(plan)
    out = torch.empty(1 << n, dtype=torch.complex64).pin_memory()
    st.download(out)
    st.sync()
    assert max_abs(out.numpy().astype(np.complex128), ref) <= TOL["c64"]
    st.close()
    plan.close()


def test_qasm_program_on_gpu():
    """A program through the OpenQASM front-end and the CUDA path equals the
    oracle on the same parsed gates (a QFT written with cu1, Toffolis and a
    user gate, 13 qubits: the dense path's smallest state)."""
    from paper_2205_06973_gb300 import qasm
    n = 13
    lines = ["OPENQASM 2.0;", 'include "qelib1.inc";', f"qreg q[{n}];", f"creg c[{n}];",
             "gate mix(a) x, y { ry(a) x; cx x, y; u3(a/2, -a, pi/3) y; }"]
    for j in range(n):
        lines.append(f"h q[{j}];")
        for m in range(1, n - j):
            lines.append(f"cu1(pi/2^{m}) q[{j + m}], q[{j}];")
    for j in range(0, n - 2, 3):
        lines.append(f"ccx q[{j}], q[{j + 1}], q[{j + 2}];")
        lines.append(f"mix({0.1 * (j + 1)}) q[{j + 2}], q[{(j + 5) % n}];")
    lines.append("measure q -> c;")
    nq, g = qasm.loads("\n".join(lines))
    assert nq == n
    psi = random_state(n, 7)
    ref = sim.run(n, g, psi)
    for prec in ("c64", "c128"):
        out = run_gpu(n, g, method="dagp", k=8, psi=psi, precision=prec)
        assert max_abs(out, ref) <= TOL[prec], prec
    out = run_gpu(n, g, method="dagp", k=6, psi=psi, tc=True)
    assert max_abs(out, ref) <= TOL["c64"]
