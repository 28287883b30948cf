"""Pins of the Hermitian-estimator oracle (Section 4), CPU."""
import numpy as np
import pytest

import oracle as O
import oracle.hermitian as OH
import synth
from oracle import rng


def test_theorems_hermitian1_and_2():
    p = synth.spectrum_exponential(40, 6.0)
    R = synth.hermitian_density(40, p, 3)
    B, C = R.real, R.imag
    assert np.allclose(B, B.T, atol=1e-15) and np.allclose(C, -C.T, atol=1e-15)
    assert np.linalg.eigvalsh(B).min() > -1e-14          # Re R is PSD
    assert abs(np.trace(R).real - np.trace(B)) < 1e-15 and abs(np.trace(R).imag) < 1e-15
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(R))[::-1], p, atol=1e-14)


@pytest.mark.parametrize("u", [1.0, 0.4])
def test_same_probe_closed_form_through_the_eigendecomposition(u):
    # g^T Re[f(R)] g = sum_i f(p_i) |psi_i^H g|^2 for real g
    n, s, m = 48, 5, 14
    p = synth.spectrum_exponential(n, 8.0)
    R = synth.hermitian_density(n, p, 4)
    G = rng.gaussian(n, s, 9)
    w, V = np.linalg.eigh(R)
    c = np.abs(V.conj().T @ G) ** 2                     # |psi_i^H g_j|^2
    a = O.cheb_coefficients(u, m)
    fm = sum(a[k] * O.cheb_T(k, w, u) for k in range(m + 1))
    ref_c = -(fm[:, None] * c).sum() / s
    assert abs(OH.chebyshev_estimate_complex(R, G, u, m) - ref_c) < 1e-12 * abs(ref_c)
    t = np.log(1 / u) + sum(((w * (1 - w / u) ** k)[:, None] * c).sum() / k
                            for k in range(1, m + 1)) / s
    assert abs(OH.taylor_estimate_complex(R, G, u, m) - t) < 1e-12 * abs(t)


def test_real_input_reduces_to_the_real_algorithms():
    n, s, m = 40, 4, 10
    R, p, _ = synth.dense_exp(n, 7.0, seed=2)
    G = rng.gaussian(n, s, 1)
    u = 0.9
    assert abs(OH.chebyshev_estimate_complex(R, G, u, m)
               - O.chebyshev_estimate_from_moments(O.chebyshev_moments(R, G, u, m), u)) < 1e-13
    assert abs(OH.taylor_estimate_complex(R, G, u, m)
               - O.taylor_estimate_from_terms(O.taylor_terms(R, G, u, m), u)) < 1e-13


def test_maximally_mixed_complex():
    # R = I/n: Taylor with u = 1 gives (1/s) sum_j |g_j|^2 sum_k (1/n)(1-1/n)^k / k
    n, s, m = 16, 3, 30
    R = np.eye(n, dtype=np.complex128) / n
    G = rng.gaussian(n, s, 2)
    k = np.arange(1, m + 1)
    ref = (G * G).sum() / s * ((1 / n) * (1 - 1 / n) ** k / k).sum()
    assert abs(OH.taylor_estimate_complex(R, G, 1.0, m) - ref) < 1e-14
