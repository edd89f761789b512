"""complex128 state-vector simulation (the "Schroedinger" approach of Sec.
"Existing Efforts on Simulation of RQCs").

Basis-state index ``i = sum_q x_q 2^q`` (qubit 0 is the least significant
bit).  Gates are applied one at a time, in circuit order, to the full
2^n-vector; the amplitude of bitstring x is then ``psi[i(x)]``.
"""
import numpy as np


def apply_1q(psi, U, q, n):
    """psi'[.., x', ..] = sum_x U[x', x] psi[.., x, ..] on qubit q."""
    v = psi.reshape(1 << (n - 1 - q), 2, 1 << q)
    return np.einsum("ij,ajb->aib", U, v).reshape(-1)


def apply_2q(psi, U, a, b, n):
    """Two-qubit gate on qubits a < b; U is indexed by 2*x_a + x_b."""
    assert a < b
    v = psi.reshape(1 << (n - 1 - b), 2, 1 << (b - 1 - a), 2, 1 << a)
    U4 = U.reshape(2, 2, 2, 2)          # [xa', xb', xa, xb]
    # v axes: h, xb, m, xa, l
    w = np.einsum("pqrs,hsmrl->hqmpl", U4, v)
    return w.reshape(-1)


def simulate(gates, n):
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for g in gates:
        if len(g.qubits) == 1:
            psi = apply_1q(psi, g.matrix, g.qubits[0], n)
        else:
            a, b = g.qubits
            psi = apply_2q(psi, g.matrix, a, b, n)
    return psi


def basis_index(bits):
    return int(sum(int(b) << q for q, b in enumerate(bits)))


def amplitudes(psi, n, bit_rows, open_qubits=()):
    """Amplitudes for each bitstring (rows of qubit values, shape (nb, n)).

    Returns complex128 (nb, 2^k): entry j sets qubit open_qubits[t] to bit t
    of j and every other qubit to the bitstring's value (open bits ignored).
    """
    k = len(open_qubits)
    bit_rows = np.asarray(bit_rows)
    out = np.empty((len(bit_rows), 1 << k), dtype=np.complex128)
    for i, bits in enumerate(bit_rows):
        b = np.array(bits, dtype=np.int64).copy()
        for j in range(1 << k):
            for t, q in enumerate(open_qubits):
                b[q] = (j >> t) & 1
            out[i, j] = psi[basis_index(b)]
    return out
