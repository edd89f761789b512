"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the simulation method: it only draws
numbers.  Everything here is a pure function of its seed, so the CUDA path and
the CPU oracle see byte-identical inputs.

* ``SplitMix64`` -- the counter-based generator of Steele, Lea and Flood,
  "Fast splittable pseudorandom number generators" (OOPSLA 2014): the state
  advances by the golden-ratio gamma and each output is the state passed
  through the two multiply-xorshift rounds of that paper.
* ``bitstrings`` -- output bitstrings of an ``n``-qubit register, packed as
  ``ceil(n/64)`` little-endian 64-bit words per bitstring (bit ``q`` of the
  word array is the value of qubit ``q``).
* ``random_tensor`` / ``random_perm`` -- the complex N(0,1) operands and index
  permutations of the pairwise-contraction microbenchmark.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
# The bitstring stream is decorrelated from the circuit stream of the same seed.
BITSTRING_STREAM_XOR = 0x9E3779B97F4A7C15


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014), 64-bit outputs as Python ints."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next(self) -> int:
        self.state = (self.state + GOLDEN_GAMMA) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)


def words_per_bitstring(n: int) -> int:
    return max(1, (n + 63) // 64)


def bitstrings(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` bitstrings of ``n`` qubits drawn from the bitstring stream.

    Qubit ``q`` of bitstring ``i`` takes the top bit of the ``(i*n + q)``-th
    draw.  Returns uint64 words, shape ``(count, ceil(n/64))``.
    """
    rng = SplitMix64(seed ^ BITSTRING_STREAM_XOR)
    w = words_per_bitstring(n)
    out = np.zeros((count, w), dtype=np.uint64)
    for i in range(count):
        for q in range(n):
            if rng.next() >> 63:
                out[i, q // 64] |= np.uint64(1) << np.uint64(q % 64)
    return out


def bits_of(words: np.ndarray, n: int) -> np.ndarray:
    """Unpack one bitstring's words into an int array of ``n`` qubit values."""
    return np.array([(int(words[q // 64]) >> (q % 64)) & 1 for q in range(n)], dtype=np.int64)


def pack_bits(bits) -> np.ndarray:
    """Inverse of :func:`bits_of` for a single bitstring."""
    n = len(bits)
    out = np.zeros(words_per_bitstring(n), dtype=np.uint64)
    for q, b in enumerate(bits):
        if int(b) & 1:
            out[q // 64] |= np.uint64(1) << np.uint64(q % 64)
    return out


def random_tensor(rank: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """A rank-``rank`` tensor with every dimension 2 and N(0,1) real and
    imaginary parts, flattened in row-major order (first index slowest)."""
    g = np.random.default_rng(seed)
    size = 1 << rank
    re = g.standard_normal(size)
    im = g.standard_normal(size)
    return (re + 1j * im).astype(dtype)


def random_perm(k: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).permutation(k)
