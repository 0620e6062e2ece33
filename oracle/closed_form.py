"""Exact results used to pin the oracle and the GPU path (test infrastructure).

* ``qft_state(psi)``: the quantum Fourier transform (the ``qft`` family of the
  paper's Table I) maps |x> to 2^{-n/2} sum_y exp(2 pi i x y / 2^n) |y>, i.e.
  it is sqrt(N) times numpy's inverse DFT of the amplitude vector.
* ``qft_basis_amplitude(n, x, y)``: one amplitude of the QFT of a basis
  state, with the phase numerator (x*y mod 2^n) kept as an exact integer.
* ``ghz(n)``: H on qubit 0 then CX(q_i, q_{i+1}) gives (|0..0> + |1..1>)/sqrt 2.
"""
from __future__ import annotations

import math

import numpy as np


def qft_state(psi: np.ndarray) -> np.ndarray:
    N = len(psi)
    return np.fft.ifft(np.asarray(psi, dtype=np.complex128)) * math.sqrt(N)


def qft_basis_amplitude(n: int, x: int, y):
    """Amplitude <y| QFT |x> for integer or integer-array y (exact phase index)."""
    N = 1 << n
    y = np.asarray(y, dtype=np.uint64)
    # uint64 products wrap modulo 2^64, and 2^n divides 2^64, so the masked
    # product is x*y mod 2^n exactly for every n <= 64
    with np.errstate(over="ignore"):
        num = (np.uint64(x % N) * y) & np.uint64(N - 1)
    ang = 2.0 * math.pi * (num.astype(np.float64) / float(N))
    return (np.cos(ang) + 1j * np.sin(ang)) * 2.0 ** (-n / 2.0)


def ghz(n: int) -> np.ndarray:
    s = np.zeros(1 << n, dtype=np.complex128)
    s[0] = s[-1] = 1.0 / math.sqrt(2.0)
    return s


def ghz_circuit(n: int):
    return [("H", (0,), 0.0)] + [("CX", (i, i + 1), 0.0) for i in range(n - 1)]
