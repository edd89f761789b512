"""Gate matrices of the benchmark gate set, complex128.

The paper names the two-qubit gate (fSim, Sec. "Searching for Better
Contraction Paths with a Reduced Complexity") but prints no matrices; the
single-qubit set {sqrt(X), sqrt(Y), sqrt(W)} is the one of the benchmark
workload.  The matrices below are the standard ones:

* sqrt(X) = (1/sqrt2) [[1, -i], [-i, 1]]          (sqrt(X)^2 = -i X)
* sqrt(Y) = (1/sqrt2) [[1, -1], [1, 1]]           (sqrt(Y)^2 = -i Y)
* sqrt(W) = (1/sqrt2) [[1, -e^{i pi/4}], [e^{-i pi/4}, 1]],  W = (X+Y)/sqrt2
* fSim(theta, phi) in the basis |x_a x_b>, index 2*x_a + x_b, a the
  lower-numbered qubit:
  [[1,0,0,0], [0,cos t,-i sin t,0], [0,-i sin t,cos t,0], [0,0,0,e^{-i phi}]]
"""
import numpy as np

_S2 = 1.0 / np.sqrt(2.0)

SQRT_X = _S2 * np.array([[1.0, -1.0j], [-1.0j, 1.0]], dtype=np.complex128)
SQRT_Y = _S2 * np.array([[1.0, -1.0], [1.0, 1.0]], dtype=np.complex128)
SQRT_W = _S2 * np.array([[1.0, -np.exp(1.0j * np.pi / 4)],
                         [np.exp(-1.0j * np.pi / 4), 1.0]], dtype=np.complex128)

ONE_QUBIT = {"sqrtx": SQRT_X, "sqrty": SQRT_Y, "sqrtw": SQRT_W}
# Draw order of the single-qubit kinds (index 0, 1, 2 of the uniform draw).
ONE_QUBIT_KINDS = ("sqrtx", "sqrty", "sqrtw")

FSIM_THETA = np.pi / 2
FSIM_PHI = np.pi / 6


def fsim(theta: float, phi: float) -> np.ndarray:
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[1, 0, 0, 0],
                     [0, c, -1j * s, 0],
                     [0, -1j * s, c, 0],
                     [0, 0, 0, np.exp(-1j * phi)]], dtype=np.complex128)
