"""Pins of the oracle's statistics: closed forms of the exponential
(Porter-Thomas) law, brute-force inverse-CDF sampling, and the physics of a
deep random circuit (Sec. "Result Validation with Different Precisions")."""
import numpy as np

from oracle import circuit as C
from oracle import stats as S
from oracle import statevector as SV


def test_porter_thomas_moments_of_exponential_law():
    n = 20
    x = np.random.default_rng(0).exponential(1.0, 400_000)
    m1, m2 = S.porter_thomas_moments(x / 2.0 ** n, n)
    assert abs(m1 - 1.0) < 0.01 and abs(m2 - 2.0) < 0.03


def test_xeb_closed_forms():
    n = 10
    uniform = np.full(1 << n, 2.0 ** -n)
    assert abs(S.exact_xeb_expectation(uniform, n)) < 1e-12
    delta = np.zeros(1 << n)
    delta[3] = 1.0
    assert abs(S.exact_xeb_expectation(delta, n) - (2.0 ** n - 1)) < 1e-9


def test_inverse_cdf_sampling_brute_force():
    p = np.array([0.5, 0.25, 0.0, 0.25])
    idx = S.sample_inverse_cdf(p, [0.0, 0.49, 0.5, 0.74, 0.75, 0.999])
    assert list(idx) == [0, 0, 1, 1, 3, 3]


def test_deep_circuit_is_porter_thomas_and_xeb_of_exact_samples():
    rows, cols, depth = 4, 4, 14
    n = rows * cols
    psi = SV.simulate(C.random_circuit(rows, cols, depth, 3), n)
    p = np.abs(psi) ** 2
    assert abs(p.sum() - 1) < 1e-12
    F = S.exact_xeb_expectation(p, n)
    assert 0.8 < F < 1.2           # Porter-Thomas gives 1
    u = np.random.default_rng(1).random(20000)
    samples = S.sample_inverse_cdf(p, u)
    f_hat = S.linear_xeb(p[samples], n)
    # sampling error of the mean of 2^n p over 2e4 draws is ~ sqrt(6)/sqrt(2e4) ~ 0.02
    assert abs(f_hat - F) < 0.1
    m1, m2 = S.porter_thomas_moments(p[np.random.default_rng(2).integers(0, 1 << n, 20000)], n)
    assert abs(m1 - 1) < 0.05 and abs(m2 - 2) < 0.3
