"""Pins of the CPU oracle's simulator against facts that do not come from it.

* gate matrices: exponentials of Pauli generators (scipy.linalg.expm) and
  projector / Pauli expansions of the 2-qubit gates (Sec. II-A conventions);
* dense 2^n x 2^n products built with Kronecker products (n <= 8);
* unitarity: the norm is preserved (Sec. II-A, U U^dagger = 1);
* GHZ state and the QFT: exact closed forms (numpy's inverse DFT);
* the index pattern of Sec. III-A / Fig. 1 (H on q0 and q1 of 3 qubits);
* Algorithm 1 (Gather-Execute-Scatter) equals gate-by-gate simulation for
  any acyclic partition and any choice of inner qubit order.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import synth
from oracle import closed_form as cf
from oracle import partition as pt
from oracle import sim

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def embed(n, ops):
    """Dense operator of a product of single-qubit operators {qubit: 2x2} on
    n qubits; little-endian index means qubit n-1 is the leftmost factor."""
    M = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        M = np.kron(M, ops.get(q, I2))
    return M


def dense_gate(n, name, qs, th):
    if name in ("H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "P"):
        u = {
            "H": (X + Z) / math.sqrt(2),
            "X": X, "Y": Y, "Z": Z,
            "S": expm(1j * math.pi / 4 * (I2 - Z)),      # diag(1, i)
            "T": expm(1j * math.pi / 8 * (I2 - Z)),      # diag(1, e^{i pi/4})
            "RX": expm(-1j * th / 2 * X),
            "RY": expm(-1j * th / 2 * Y),
            "RZ": expm(-1j * th / 2 * Z),
            "P": expm(1j * th / 2 * (I2 - Z)),           # diag(1, e^{i th})
        }[name]
        return embed(n, {qs[0]: u})
    c, t = qs
    if name == "CX":
        return embed(n, {c: P0}) + embed(n, {c: P1, t: X})
    if name == "CZ":
        return embed(n, {}) - 2 * embed(n, {c: P1, t: P1})
    if name == "CP":
        return embed(n, {}) + (np.exp(1j * th) - 1) * embed(n, {c: P1, t: P1})
    if name == "SWAP":
        return 0.5 * (embed(n, {}) + embed(n, {c: X, t: X}) + embed(n, {c: Y, t: Y})
                      + embed(n, {c: Z, t: Z}))
    raise ValueError(name)


def random_circuit(n, G, seed):
    r = synth.SplitMix64(seed)
    gates = []
    for _ in range(G):
        name = synth.GATE_NAMES[r.randint(len(synth.GATE_NAMES))]
        if name in synth.TWO_QUBIT:
            if n < 2:
                continue
            a = r.randint(n)
            b = (a + 1 + r.randint(n - 1)) % n
            qs = (a, b)
        else:
            qs = (r.randint(n),)
        gates.append((name, qs, r.angle()))
    return gates


def random_state(n, seed):
    a = synth.random_amplitudes(n, seed)
    v = a[:, 0] + 1j * a[:, 1]
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("name", synth.GATE_NAMES)
def test_gate_matrix_matches_generator_form(name):
    th = 0.7319
    n = 3
    qs = (1,) if name in synth.ONE_QUBIT else (2, 0)
    D = dense_gate(n, name, qs, th)
    for x in range(1 << n):
        out = sim.run(n, [(name, qs, th)], sim.basis(n, x))
        assert np.abs(out - D[:, x]).max() < 1e-14, (name, x)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_dense_unitary_product(n):
    gates = random_circuit(n, 40, seed=100 + n)
    U = np.eye(1 << n, dtype=complex)
    for name, qs, th in gates:
        U = dense_gate(n, name, qs, th) @ U
    psi = random_state(n, 7 + n)
    out = sim.run(n, gates, psi)
    assert np.abs(out - U @ psi).max() < 1e-13


def test_norm_preserved_and_probs():
    n = 12
    gates = random_circuit(n, 300, seed=3)
    out = sim.run(n, gates, random_state(n, 4))
    p, tot = sim.probs(out)
    assert abs(tot - 1.0) < 1e-12
    assert np.allclose(p, np.abs(out) ** 2, atol=0, rtol=1e-15)


@pytest.mark.parametrize("n", [2, 5, 11])
def test_ghz(n):
    out = sim.run(n, cf.ghz_circuit(n))
    assert np.abs(out - cf.ghz(n)).max() < 1e-15


@pytest.mark.parametrize("n", [1, 3, 6, 10])
def test_qft_is_inverse_dft(n):
    psi = random_state(n, 11 + n)
    out = sim.run(n, synth.qft(n), psi)
    assert np.abs(out - cf.qft_state(psi)).max() < 1e-13


def test_qft_basis_closed_form():
    n = 13
    x = synth.SplitMix64(3).randint(1 << n)
    out = sim.run(n, synth.qft(n), sim.basis(n, x))
    ref = cf.qft_basis_amplitude(n, x, np.arange(1 << n))
    assert np.abs(out - ref).max() < 1e-13


def test_qft_gate_count_33():
    n, g, x = synth.qft_basis(33)
    assert len(g) == 33 + 528 + 16


def test_index_pattern_of_fig1():
    """H on q0 pairs (a000, a001), ...; H on q1 pairs elements at stride 2."""
    n = 3
    for q in (0, 1):
        for x in range(8):
            out = sim.run(n, [("H", (q,), 0.0)], sim.basis(n, x))
            nz = set(np.flatnonzero(np.abs(out) > 1e-12).tolist())
            assert nz == {x, x ^ (1 << q)}


def test_alg1_single_part_example():
    """Algorithm 1 walk-through: part P0 on {q1, q0} of 4 qubits runs its
    gates on 4-element inner vectors for each of the 4 values of (q3, q2)."""
    n = 4
    gates = [("H", (1,), 0.0), ("CX", (1, 0), 0.0), ("RZ", (0,), 0.4)]
    psi = random_state(n, 5)
    a = sim.run(n, gates, psi)
    b = sim.run_alg1(n, gates, [0, 0, 0], 1, psi)
    assert np.abs(a - b).max() < 1e-15
    # the same result is reached by applying the 4x4 part unitary to each
    # gathered quadruple (q3, q2 fixed)
    U = np.eye(4, dtype=complex)
    for name, qs, th in gates:
        U = dense_gate(2, name, qs, th) @ U
    c = psi.copy()
    for hi in range(4):
        idx = [hi * 4 + l for l in range(4)]
        c[idx] = U @ psi[idx]
    assert np.abs(a - c).max() < 1e-15


@pytest.mark.parametrize("method", ["nat", "dfs", "dagp"])
@pytest.mark.parametrize("k", [2, 3, 5])
def test_alg1_equals_gatewise(method, k):
    n = 9
    gates = random_circuit(n, 120, seed=20 + k)
    pog = pt.partition(gates, n, method, k, seed=9)
    P = pt.check_partition(gates, n, k, pog)
    psi = random_state(n, 21)
    a = sim.run(n, gates, psi)
    b = sim.run_alg1(n, gates, pog, P, psi)
    c = sim.run_alg1(n, gates, pog, P, psi, order_mode=1)
    assert np.abs(a - b).max() < 1e-13
    assert np.abs(a - c).max() < 1e-13


def test_workload_generators_shape():
    n, g = synth.plain_layered_14q()
    assert n == 14 and len(g) == 840
    n, g = synth.layered_28q()
    assert n == 28 and len(g) == 2520
    names = synth.gate_count_by_name(g)
    assert set(names) == {"H", "RX", "RZ", "CX", "CZ"}
    ns = [synth.batch_circuit(i)[0] for i in range(200)]
    assert min(ns) >= 10 and max(ns) <= 20
