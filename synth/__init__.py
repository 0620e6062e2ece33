"""Seeded synthetic circuit generators.

This module is shared by the CPU oracle and the GPU path. It holds no
simulation arithmetic: it only draws gate lists, angles, qubit counts and
arrival times from a SplitMix64 stream. A gate is a tuple
``(name, qubits, theta)`` where ``name`` is one of ``GATE_NAMES``, ``qubits``
is a tuple of qubit indices (for controlled gates the control comes first)
and ``theta`` is the rotation/phase angle in radians (0.0 when unused).
Each consumer maps the names onto its own gate codes.

The workloads stand in for the QASMBench circuits of the paper's Table I,
which are not available here:

* ``layered``   - random layered circuits: one gate from a 1-qubit set on
  every qubit, then a 2-qubit gate on each pair of a random disjoint pairing.
* ``qft``       - the quantum Fourier transform network (H, controlled-phase
  ladders, final swaps), the ``qft`` family of Table I.
* ``param``     - parameterised ansatz layers: RY and RZ on every qubit then a
  CX ladder.
* ``batch_circuits`` / ``serving_stream`` - many independent circuits and a
  Poisson request stream built from the three families.
"""
from __future__ import annotations

import math

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

ONE_QUBIT = ("H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "P")
TWO_QUBIT = ("CX", "CZ", "CP", "SWAP")
GATE_NAMES = ONE_QUBIT + TWO_QUBIT
PARAMETRIC = ("RX", "RY", "RZ", "P", "CP")


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): a Weyl counter with
    increment 0x9E3779B97F4A7C15 passed through a 64-bit finaliser."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + GOLDEN) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def randint(self, m: int) -> int:
        """Integer in [0, m) as next() mod m."""
        return self.next() % m

    def angle(self) -> float:
        return self.uniform() * 2.0 * math.pi

    def permutation(self, n: int) -> list[int]:
        """Fisher-Yates shuffle of 0..n-1 (i from n-1 down to 1, j = randint(i+1))."""
        p = list(range(n))
        for i in range(n - 1, 0, -1):
            j = self.randint(i + 1)
            p[i], p[j] = p[j], p[i]
        return p


def layered(n: int, depth: int, seed: int, one_q=("H", "RX", "RZ"),
            two_q=("CX",), rng: SplitMix64 | None = None):
    """Random layered circuit.

    Each layer: for qubit q = 0..n-1 draw a gate from ``one_q`` (randint) and,
    if it is parametric, an angle uniform in [0, 2*pi); then a Fisher-Yates
    permutation pi of 0..n-1 pairs (pi[0], pi[1]), (pi[2], pi[3]), ... with
    the first element as control; with more than one 2-qubit kind each pair
    draws its kind with randint(len(two_q)). Odd n leaves one qubit idle.
    """
    r = rng if rng is not None else SplitMix64(seed)
    gates = []
    for _ in range(depth):
        for q in range(n):
            name = one_q[r.randint(len(one_q))]
            th = r.angle() if name in PARAMETRIC else 0.0
            gates.append((name, (q,), th))
        pi = r.permutation(n)
        for i in range(n // 2):
            name = two_q[r.randint(len(two_q))] if len(two_q) > 1 else two_q[0]
            th = r.angle() if name in PARAMETRIC else 0.0
            gates.append((name, (pi[2 * i], pi[2 * i + 1]), th))
    return gates


def qft(n: int):
    """QFT network: for j = n-1 down to 0, H on q_j followed by CP(pi/2^m)
    with control q_{j-m} and target q_j for m = 1..j; then SWAP(q_i, q_{n-1-i})
    for i < n/2. Maps |x> to 2^{-n/2} sum_y exp(2 pi i x y / 2^n) |y>."""
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(("H", (j,), 0.0))
        for m in range(1, j + 1):
            gates.append(("CP", (j - m, j), math.pi / (1 << m)))
    for i in range(n // 2):
        gates.append(("SWAP", (i, n - 1 - i), 0.0))
    return gates


def param(n: int, depth: int, seed: int, rng: SplitMix64 | None = None):
    """Parameterised layers: RY(theta) on every qubit, then RZ(theta) on every
    qubit, then CX(i, i+1) for i = 0..n-2; angles uniform in [0, 2*pi)."""
    r = rng if rng is not None else SplitMix64(seed)
    gates = []
    for _ in range(depth):
        for q in range(n):
            gates.append(("RY", (q,), r.angle()))
        for q in range(n):
            gates.append(("RZ", (q,), r.angle()))
        for q in range(n - 1):
            gates.append(("CX", (q, q + 1), 0.0))
    return gates


# --- the five workloads -----------------------------------------------------

def plain_layered_14q():
    """14 qubits, depth 40, {H, RX, RZ} then CX pairs: 40 * (14 + 7) = 840 gates, seed 1."""
    return 14, layered(14, 40, seed=1, one_q=("H", "RX", "RZ"), two_q=("CX",))


def layered_28q(n: int = 28, depth: int = 60, seed: int = 2):
    """28 qubits, depth 60, {H, RX, RZ} then CX/CZ pairs: 60 * 42 = 2520 gates, seed 2."""
    return n, layered(n, depth, seed=seed, one_q=("H", "RX", "RZ"), two_q=("CX", "CZ"))


def qft_basis(n: int = 33, seed: int = 3):
    """QFT on n qubits applied to a seeded basis state |x>, x uniform in [0, 2^n)."""
    x = SplitMix64(seed).randint(1 << n)
    return n, qft(n), x


def batch_circuit(i: int):
    """Circuit i of the batched workload: seed 4*2^32 + i; n uniform in
    10..20, depth uniform in 10..50, then the ``param`` layers."""
    r = SplitMix64((4 << 32) + i)
    n = 10 + r.randint(11)
    depth = 10 + r.randint(41)
    return n, param(n, depth, seed=0, rng=r)


def batch_circuits(count: int = 4096, start: int = 0):
    return [batch_circuit(i) for i in range(start, start + count)]


def serving_request(i: int, seed: int = 5):
    """Request i of the serving stream (circuit only; arrival times come from
    ``serving_arrivals``). With probability 0.8, n ~ U{10..20}, else
    U{21..33}; family uniform over layered (depth U{10..40}), qft and param
    (depth U{10..50})."""
    r = SplitMix64((seed << 32) + i)
    if r.uniform() < 0.8:
        n = 10 + r.randint(11)
    else:
        n = 21 + r.randint(13)
    fam = ("layered", "qft", "param")[r.randint(3)]
    if fam == "layered":
        d = 10 + r.randint(31)
        g = layered(n, d, seed=0, one_q=("H", "RX", "RZ"), two_q=("CX", "CZ"), rng=r)
    elif fam == "qft":
        g = qft(n)
    else:
        d = 10 + r.randint(41)
        g = param(n, d, seed=0, rng=r)
    return n, fam, g


def serving_arrivals(count: int = 20000, duration_s: float = 60.0, seed: int = 5):
    """Poisson arrival times: exponential gaps with rate count/duration."""
    r = SplitMix64(seed)
    lam = count / duration_s
    t = 0.0
    out = []
    for _ in range(count):
        t += -math.log(1.0 - r.uniform()) / lam
        out.append(t)
    return out


def splitmix_block(seed: int, start: int, count: int):
    """Outputs start..start+count-1 of SplitMix64(seed) as a numpy uint64
    array. SplitMix64 is counter based: output i (0-based) is the finaliser
    applied to seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64)."""
    import numpy as np
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + i * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def random_amplitudes(n: int, seed: int):
    """2^n unnormalised complex amplitudes with real and imaginary parts
    uniform in [-1, 1): element x takes outputs 2x (real) and 2x+1 (imag).
    Returned as a float64 array of shape (2^n, 2); callers normalise with
    their own arithmetic."""
    import numpy as np
    z = splitmix_block(seed, 0, 2 << n)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return (2.0 * u - 1.0).reshape(1 << n, 2)


def gate_count_by_name(gates):
    out = {}
    for g in gates:
        out[g[0]] = out.get(g[0], 0) + 1
    return out
