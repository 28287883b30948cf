"""Pins of the learned-correction oracle (CPU)."""
import numpy as np
import pytest

import oracle as O
import oracle.learned as L
import synth
from oracle import rng


def test_spectral_totals_equal_algorithm_1b_moments_on_the_matrix():
    # R = Psi diag(p) Psi^T with probes G = Psi Z: the forward-recurrence
    # moments of Algorithm 1b summed over probes equal the spectral totals
    n, s, m, seed = 64, 5, 12, 7
    psi = synth.haar_orthogonal(n, 3)
    p = synth.spectrum_exponential(n, 9.0)
    R = synth.dense_density(psi, p)
    u = 1.05 * p.max()
    Z = rng.gaussian(n, s, seed)
    mu = O.chebyshev_moments(R, psi @ Z, u, m)
    tot = L.spectral_totals(p, u, m, s, seed)
    np.testing.assert_allclose(tot, mu.sum(axis=1), rtol=1e-10, atol=1e-10 * np.abs(tot).max())
    H = L.chebyshev_from_totals(tot, u, s)
    assert abs(H - O.chebyshev_estimate_from_moments(mu, u)) < 1e-12


def test_expected_totals_give_the_exact_polynomial_trace():
    # E[sum_j z_ij^2] = s: replacing w_i by s gives -tr f_m(R) (NTE)
    n, s, m = 200, 8, 16
    p = synth.training_spectrum(1, n, 1.5, 50, 1e-8)
    u = p.max()
    x = 2 * p / u - 1
    tot = s * np.polynomial.chebyshev.chebvander(x, m).sum(axis=0)
    assert abs(L.chebyshev_from_totals(tot, u, s) - O.nte_chebyshev(p, u, m)) < 1e-12


def test_target_of_uniform_spectrum():
    n = 128
    p = np.full(n, 1.0 / n)
    assert abs(L.entropy(p) - np.log(n)) < 1e-13
    assert abs(L.target(p, np.log(n) - 0.5, 2.0 / n) - 100 * 0.5 / 2.0) < 1e-11


def test_target_is_the_truncation_error_over_n_u():
    # with w_i = s exactly, H - H_m = -u sum_i e_m(p_i / u): the target is
    # -100 * mean_i e_m(y_i) for any n with the same distribution of y
    m, s = 16, 4
    for n in (256, 4096):
        y = (np.arange(n) + 0.5) / n  # the same distribution of y = p/u at both sizes
        p = y / y.sum()
        u = p.max() / y.max()
        tot = s * np.polynomial.chebyshev.chebvander(2 * p / u - 1, m).sum(axis=0)
        t = L.target(p, L.chebyshev_from_totals(tot, u, s), u)
        e = y * np.log(y) - O.cheb_fm(y, 1.0, m)
        assert abs(t - (-100.0 * e.mean())) < 1e-9 * max(1.0, abs(t))


def test_gelu_values():
    assert L.gelu(0.0) == 0.0
    assert abs(L.gelu(10.0) - 10.0) < 1e-12 and abs(L.gelu(-10.0)) < 1e-12
    assert abs(L.gelu_grad(0.0) - 0.5) < 1e-15
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    np.testing.assert_allclose(L.gelu_grad(x), (L.gelu(x + h) - L.gelu(x - h)) / (2 * h),
                               rtol=1e-7, atol=1e-9)


def test_zero_weights_output_last_bias():
    theta = np.zeros(L.N_PARAMS)
    theta[-1] = 0.25
    y, _ = L.forward(theta, np.random.default_rng(0).standard_normal((7, L.N_IN)))
    np.testing.assert_array_equal(y, np.full(7, 0.25))


def test_backward_matches_central_differences():
    rs = np.random.default_rng(1)
    theta = synth.mlp_init(5)
    X = rs.standard_normal((16, L.N_IN))
    t = rs.standard_normal(16) * 0.1
    loss, g = L.backward(theta, X, t)
    assert abs(loss - L.mse(L.forward(theta, X)[0], t)) < 1e-15
    idx = np.concatenate([rs.choice(L.N_PARAMS, 60, replace=False),
                          [0, L.N_PARAMS - 1, L.N_PARAMS - 2]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (L.mse(L.forward(tp, X)[0], t) - L.mse(L.forward(tm, X)[0], t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, np.abs(g).max()), (i, fd, g[i])


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th, m, v = L.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    np.testing.assert_allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


@pytest.mark.parametrize("kind", [0, 1])
def test_training_spectra_are_density_spectra(kind):
    p = synth.training_spectrum(kind, 1500, 200.0 if kind == 0 else 1.4, 300, 1e-9)
    assert abs(p.sum() - 1.0) < 1e-12 and np.all(p > 0) and np.all(np.diff(p) <= 0)
    # eigh of the assembled matrix returns the same spectrum (labels are exact)
    n = 96
    q = synth.training_spectrum(kind, n, 20.0 if kind == 0 else 1.4, 30, 1e-9)
    R = synth.dense_density(synth.haar_orthogonal(n, 2), q)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(R))[::-1], q, atol=1e-15)
