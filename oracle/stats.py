"""Statistics of output probabilities (Sec. "Result Validation with Different
Precisions": Porter-Thomas; Appendix A: linear cross-entropy benchmark).

For an n-qubit chaotic random circuit the rescaled probabilities
``x = 2^n p`` follow the Porter-Thomas law with density e^{-x}: E[x] = 1 over
uniformly drawn bitstrings and E[x^2] = 2.  The linear XEB of samples drawn
from the circuit's own output distribution is F = 2^n <p(x_i)> - 1, which
equals 2^n sum_x p(x)^2 - 1 in expectation (= 1 for Porter-Thomas).
"""
import numpy as np


def porter_thomas_moments(p, n):
    x = (2.0 ** n) * np.asarray(p, dtype=np.float64)
    return float(np.mean(x)), float(np.mean(x * x))


def linear_xeb(p_of_samples, n):
    return float((2.0 ** n) * np.mean(np.asarray(p_of_samples, dtype=np.float64)) - 1.0)


def exact_xeb_expectation(p_all, n):
    """E[F] over exact samples: 2^n sum_x p(x)^2 - 1."""
    p = np.asarray(p_all, dtype=np.float64)
    return float((2.0 ** n) * np.sum(p * p) - 1.0)


def sample_inverse_cdf(p_all, u):
    """Draw one basis index per uniform u in [0, 1) from distribution p_all
    by inverting its cumulative sum (the uniforms are passed in)."""
    c = np.cumsum(np.asarray(p_all, dtype=np.float64))
    c /= c[-1]
    return np.searchsorted(c, np.asarray(u, dtype=np.float64), side="right")
