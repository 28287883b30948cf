"""Pins of the oracle's Chebyshev expansion of h(x) = x ln x (CPU only).

Lemma lem:prior fixes the coefficients and the uniform error bound
u / (2m(m+1)); a library Chebyshev interpolation of h (NumPy) and the
library evaluator ``chebval`` are independent checks of both.
"""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as C

import oracle as O


def h(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    pos = x > 0
    out[pos] = x[pos] * np.log(x[pos])
    return out


@pytest.mark.parametrize("u", [1.0, 0.7, 0.0198, 0.39])
def test_coefficients_match_library_interpolant(u):
    # Chebyshev interpolant of h(u (t + 1) / 2) on [-1, 1] at high degree;
    # its aliasing error is O(u / N^3).
    N = 2000
    ref = C.chebinterpolate(lambda t: h(u * (t + 1.0) / 2.0), N)
    a = O.cheb_coefficients(u, 30)
    np.testing.assert_allclose(a, ref[:31], rtol=0, atol=1e-9 * u)


def test_coefficients_printed_form_u07():
    a = O.cheb_coefficients(0.7, 3)
    # (u/2)(ln(u/4)+1), (u/4)(2 ln(u/4)+3), u/6, -u/24 at u = 0.7
    np.testing.assert_allclose(a, [-0.26003926, -0.08503926, 0.11666667, -0.02916667],
                               atol=5e-9)


@pytest.mark.parametrize("u,m", [(1.0, 5), (0.7, 20), (0.7, 40), (0.02, 13)])
def test_uniform_error_bound_and_where_attained(u, m):
    x = np.linspace(0.0, u, 200_001)
    err = np.abs(h(x) - O.cheb_fm(x, u, m))
    bound = u / (2.0 * m * (m + 1))
    assert err.max() <= bound * (1 + 1e-9)
    # the bound is attained at x = 0, where h(0) = 0 and f_m(0) = -bound
    np.testing.assert_allclose(O.cheb_fm(np.array([0.0]), u, m)[0], -bound, rtol=1e-11)
    np.testing.assert_allclose(err.max(), bound, rtol=1e-9)


@pytest.mark.parametrize("m", [0, 1, 2, 7, 30])
def test_fm_matches_library_chebval(m):
    u = 0.31
    x = np.linspace(-0.05, u + 0.05, 1001)  # also just outside [0, u]
    a = O.cheb_coefficients(u, m)
    ref = C.chebval((2.0 / u) * x - 1.0, a)
    np.testing.assert_allclose(O.cheb_fm(x, u, m), ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("m", [0, 1, 2, 3, 12])
def test_clenshaw_scalar_equals_fm(m):
    # R = diag(x), g = e_i gives g^T f_m(R) g = f_m(x_i) (Appendix C)
    u = 0.5
    x = np.array([0.0, 1e-6, 0.1, 0.25, 0.49, 0.5])
    R = np.diag(x)
    G = np.eye(len(x))
    got = O.clenshaw_quadforms(R, G, u, m)
    np.testing.assert_allclose(got, O.cheb_fm(x, u, m), rtol=1e-12, atol=1e-15)


def test_suggest_m_theorems():
    # Theorem thm:taylor: m = ceil((u/l) ln(1/eps)); Theorem thm:cheb: the
    # square root, rounded up.
    assert O.suggest_m("taylor", 0.5, 0.01, 0.1) == int(np.ceil(50 * np.log(10)))
    m = O.suggest_m("chebyshev", 0.5, 0.01, 0.1)
    assert m == int(np.ceil(np.sqrt(0.5 / (2 * 0.1 * 0.01 * np.log(1 / 0.99)))))
