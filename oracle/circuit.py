"""Seeded random-circuit protocol (the oracle's own generator).

Layout (the paper's "(1+d+1)" depth notation, Sec. "Performance Attributes"):
one layer of single-qubit gates, then ``depth`` cycles, each an fSim layer on
coupler pattern ``P[c mod 4]`` followed by a single-qubit layer; the register
starts in |0...0> and is read out in the computational basis.

Coupler patterns on an R x C grid, qubit (r, c) = r*C + c:
A horizontal (r,c)-(r,c+1) with c even; B horizontal with c odd;
C vertical (r,c)-(r+1,c) with r even; D vertical with r odd; cycle A,B,C,D.

Randomness: SplitMix64 (Steele, Lea, Flood 2014) seeded with ``seed``.  A
uniform draw over ``k`` options takes ``((x >> 32) * k) >> 32`` of the next
output ``x``.  Layer 0 draws each qubit's kind from the three kinds; later
layers draw from the two kinds that differ from that qubit's previous kind;
draws go in qubit order within a layer.  fSim gates carry no randomness.
"""
from dataclasses import dataclass, field

import numpy as np

from . import gates as G

_MASK = (1 << 64) - 1


class _SplitMix64:
    def __init__(self, seed):
        self.s = seed & _MASK

    def next(self):
        self.s = (self.s + 0x9E3779B97F4A7C15) & _MASK
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, k):
        return ((self.next() >> 32) * k) >> 32


@dataclass
class Gate:
    kind: str            # "sqrtx" | "sqrty" | "sqrtw" | "fsim" | "mat1" | "mat2"
    qubits: tuple        # (q,) or (a, b) with a < b for fsim
    theta: float = 0.0
    phi: float = 0.0
    matrix: np.ndarray = field(default=None, repr=False)


def coupler_pattern(rows, cols, p):
    """Qubit pairs (a, b), a < b, of pattern p in {0:A, 1:B, 2:C, 3:D}."""
    pairs = []
    if p in (0, 1):
        for r in range(rows):
            for c in range(p, cols - 1, 2):
                pairs.append((r * cols + c, r * cols + c + 1))
    else:
        for r in range(p - 2, rows - 1, 2):
            for c in range(cols):
                pairs.append((r * cols + c, (r + 1) * cols + c))
    return pairs


def random_circuit(rows, cols, depth, seed, theta=G.FSIM_THETA, phi=G.FSIM_PHI):
    n = rows * cols
    rng = _SplitMix64(seed)
    prev = [None] * n
    out = []

    def one_qubit_layer():
        for q in range(n):
            if prev[q] is None:
                kind = G.ONE_QUBIT_KINDS[rng.uniform(3)]
            else:
                opts = [k for k in G.ONE_QUBIT_KINDS if k != prev[q]]
                kind = opts[rng.uniform(2)]
            prev[q] = kind
            out.append(Gate(kind, (q,), matrix=G.ONE_QUBIT[kind]))

    one_qubit_layer()
    fs = G.fsim(theta, phi)
    for c in range(depth):
        for a, b in coupler_pattern(rows, cols, c % 4):
            out.append(Gate("fsim", (a, b), theta, phi, fs))
        one_qubit_layer()
    return out
