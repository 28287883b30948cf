"""Pins of the oracle's estimators against closed forms, special cases,
brute force and invariants (CPU only).

Each check is chosen so that a plausible slip in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a missing 1/k) makes
one of them fail; ``test_planted_mistakes_are_caught`` plants a few such
slips in the oracle on the CPU and shows that they are.
"""
import numpy as np
import pytest
from scipy import stats

import oracle as O
import synth
from oracle import rng


def _spd(n, seed, spectrum=None):
    psi = synth.haar_orthogonal(n, seed)
    p = spectrum if spectrum is not None else synth.spectrum_exponential(n, n / 5.0)
    return synth.dense_density(psi, p), p, psi


# --- same-probe closed forms through the eigendecomposition -------------

@pytest.mark.parametrize("m", [1, 2, 3, 10, 25])
@pytest.mark.parametrize("uscale", [1.0, 1.3, 6.0])
def test_chebyshev_same_probe_spectral_closed_form(m, uscale):
    n, s = 48, 7
    R, p, psi = _spd(n, 5)
    u = min(1.0, uscale * p.max())
    G = rng.gaussian(n, s, 21)
    proj2 = (psi.T @ G) ** 2  # (psi_i^T g_j)^2
    fm = O.cheb_fm(p, u, m)
    ref_per_probe = (fm[:, None] * proj2).sum(axis=0)
    np.testing.assert_allclose(O.clenshaw_quadforms(R, G, u, m), ref_per_probe,
                               rtol=1e-11, atol=1e-14)
    mu = O.chebyshev_moments(R, G, u, m)
    a = O.cheb_coefficients(u, m)
    np.testing.assert_allclose((a[:, None] * mu).sum(axis=0), ref_per_probe,
                               rtol=1e-11, atol=1e-14)
    for k in range(m + 1):
        Tk = O.cheb_T(k, p, u)
        np.testing.assert_allclose(mu[k], (Tk[:, None] * proj2).sum(axis=0),
                                   rtol=1e-10, atol=1e-12)
    H1 = O.chebyshev_estimate_clenshaw(R, G, u, m)
    H2 = O.chebyshev_estimate_from_moments(mu, u)
    assert abs(H1 - H2) <= 1e-12 * abs(H1)


@pytest.mark.parametrize("m", [1, 2, 5, 30])
def test_taylor_same_probe_spectral_closed_form(m):
    n, s = 40, 6
    R, p, psi = _spd(n, 8)
    u = 1.2 * p.max()
    G = rng.rademacher(n, s, 4)
    proj2 = (psi.T @ G) ** 2
    tau = O.taylor_terms(R, G, u, m)
    for k in range(m + 1):
        ref = ((p * (1.0 - p / u) ** k)[:, None] * proj2).sum(axis=0)
        np.testing.assert_allclose(tau[k], ref, rtol=1e-11, atol=1e-15)
    ks = np.arange(1, m + 1)
    Href = np.log(1 / u) + sum(
        ((p * (1 - p / u) ** k)[:, None] * proj2).sum(axis=0) / k for k in ks).mean()
    assert abs(O.taylor_estimate_from_terms(tau, u) - Href) < 1e-12


# --- special cases ---------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 17, 64])
def test_maximally_mixed(n):
    R = np.eye(n) / n
    assert abs(O.exact_entropy(R) - np.log(n)) < 1e-12
    lam, _ = O.power_method(R, rng.power_start(n, 1, 3), 5)
    assert abs(lam - 1.0 / n) < 1e-15
    u = 1.0 / n
    G = rng.gaussian(n, 9, 2)
    # C = I - R/u = 0: the Taylor estimate is exactly ln n for any probes
    Ht = O.taylor_estimate_from_terms(O.taylor_terms(R, G, u, 12), u)
    assert abs(Ht - np.log(n)) < 1e-13
    # Rademacher probes: g^T g = n, so the Chebyshev estimate is -n f_m(1/n)
    Gr = rng.rademacher(n, 5, 2)
    m = 9
    Hc = O.chebyshev_estimate_clenshaw(R, Gr, u, m)
    assert abs(Hc + n * O.cheb_fm(np.array([1.0 / n]), u, m)[0]) < 1e-12
    assert abs(Hc - np.log(n)) <= n * u / (2 * m * (m + 1)) + 1e-12


def test_pure_state():
    n = 30
    psi = synth.haar_orthogonal(n, 1)[:, :1]
    R = psi @ psi.T
    assert abs(O.exact_entropy(R)) < 1e-12
    lam, _ = O.power_method(R, rng.power_start(n, 1, 5), 3)
    assert abs(lam - 1.0) < 1e-12
    G = rng.gaussian(n, 4, 1)
    # u = 1: R C = R - R^2 = 0, so every Taylor term vanishes
    Ht = O.taylor_estimate_from_terms(O.taylor_terms(R, G, 1.0, 8), 1.0)
    assert abs(Ht) < 1e-12


def test_diagonal_matrix():
    d = synth.spectrum_exponential(25, 4.0)[::-1].copy()
    R = np.diag(d)
    assert abs(O.exact_entropy(R) - stats.entropy(d)) < 1e-13
    assert abs(O.entropy_of_spectrum(d) - stats.entropy(d)) < 1e-13
    # power method from a +-1 vector: Rayleigh quotient of R^t x_0 is
    # sum d^(2t+1) / sum d^(2t)
    t = 7
    lam, _ = O.power_method(R, rng.power_start(25, 1, 9), t)
    assert abs(lam - (d ** (2 * t + 1)).sum() / (d ** (2 * t)).sum()) < 1e-15
    u, m = d.max(), 6
    G = rng.gaussian(25, 3, 8)
    ref = -(O.cheb_fm(d, u, m)[:, None] * G ** 2).sum() / 3
    assert abs(O.chebyshev_estimate_clenshaw(R, G, u, m) - ref) < 1e-13


def test_poisson_closed_form_spectrum():
    n = 300
    vals = synth.band_poisson(n)
    dense = synth.dia_to_dense(vals)
    w = np.sort(np.linalg.eigvalsh(dense))
    np.testing.assert_allclose(w, np.sort(synth.spectrum_poisson(n)), rtol=0, atol=1e-15)
    assert abs(O.exact_entropy(O.Dia(vals)) -
               O.entropy_of_spectrum(synth.spectrum_poisson(n))) < 1e-11


def test_dia_apply_matches_dense():
    vals = synth.band_diag_dominant(70, half_bw=16, seed=2, dtype=np.float64)
    dense = synth.dia_to_dense(vals)
    Y = rng.gaussian(70, 3, 1)
    np.testing.assert_allclose(O.apply_R(O.Dia(vals), Y), dense @ Y, rtol=1e-13, atol=1e-17)
    assert abs(O.trace_of(O.Dia(vals)) - 1.0) < 1e-12
    # diagonal dominance => SPD
    assert np.linalg.eigvalsh(dense).min() > 0


# --- brute force -----------------------------------------------------------

def _jacobi_eigenvalues(A, sweeps=60):
    """Cyclic Jacobi rotations (own code) for symmetric A."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    for _ in range(sweeps):
        off = np.sqrt((A ** 2).sum() - (np.diag(A) ** 2).sum())
        if off < 1e-300:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if A[p, q] == 0.0:
                    continue
                theta = (A[q, q] - A[p, p]) / (2.0 * A[p, q])
                t = np.sign(theta) / (abs(theta) + np.sqrt(theta * theta + 1.0)) if theta != 0 else 1.0
                c = 1.0 / np.sqrt(t * t + 1.0)
                s = t * c
                J = np.eye(n)
                J[p, p] = J[q, q] = c
                J[p, q] = s
                J[q, p] = -s
                A = J.T @ A @ J
    return np.sort(np.diag(A))


@pytest.mark.parametrize("n", [2, 5, 16])
def test_exact_entropy_against_jacobi(n):
    R, p, _ = _spd(n, 10 + n)
    w = _jacobi_eigenvalues(R)
    np.testing.assert_allclose(w, np.sort(p), rtol=0, atol=1e-13)
    assert abs(O.exact_entropy(R) - O.entropy_of_spectrum(w)) < 1e-13
    assert abs(O.exact_entropy(R) - O.entropy_of_spectrum(p)) < 1e-12


# --- truncation bounds of the paper ---------------------------------------

def test_taylor_identity_lemma1a():
    p = synth.spectrum_exponential(200, 30.0)
    H = O.entropy_of_spectrum(p)
    u = p.max()
    ell = p.min()
    for m in (50, 400, 3000):
        nte = O.nte_taylor(p, u, m)
        # tail of Lemma lem1a: |NTE - H| <= sum_{k>m} tr(R C^k)/k <= (1-l/u)^m H
        # (the last step of the proof of Theorem thm:taylor)
        assert 0.0 <= H - nte <= (1 - ell / u) ** m * H + 1e-12


@pytest.mark.parametrize("m", [5, 20, 40])
def test_chebyshev_nte_within_pd2(m):
    p = synth.spectrum_exponential(512, 50.0)
    H = O.entropy_of_spectrum(p)
    u = p.max()
    nte = O.nte_chebyshev(p, u, m)
    assert abs(nte - H) <= len(p) * u / (2 * m * (m + 1))  # eq. PD2


# --- trace-estimator invariants ---------------------------------------------

def test_hutchinson_linearity_and_probe_partition():
    n = 33
    R, p, _ = _spd(n, 2)
    u, m = 1.1 * p.max(), 8
    G = rng.gaussian(n, 10, 3)
    G1, G2 = G[:, :4], G[:, 4:]
    H = O.chebyshev_estimate_clenshaw(R, G, u, m)
    H1 = O.chebyshev_estimate_clenshaw(R, G1, u, m)
    H2 = O.chebyshev_estimate_clenshaw(R, G2, u, m)
    assert abs(H - (4 * H1 + 6 * H2) / 10) < 1e-13
    mu = O.chebyshev_moments(R, G, u, m)
    perm = np.array([7, 2, 9, 0, 1, 5, 3, 8, 6, 4])
    np.testing.assert_allclose(O.chebyshev_moments(R, G[:, perm], u, m), mu[:, perm],
                               rtol=1e-13, atol=1e-14)


def test_hutchinson_unbiased_within_5_sigma():
    n, s = 30, 4000
    R, p, _ = _spd(n, 6)
    u, m = p.max(), 10
    nte = O.nte_chebyshev(p, u, m)
    a = -O.cheb_fm(p, u, m)
    sigma = np.sqrt(2 * (a ** 2).sum() / s)  # Gaussian quadratic-form variance
    Hc = O.chebyshev_estimate_clenshaw(R, rng.gaussian(n, s, 77), u, m)
    assert abs(Hc - nte) < 5 * sigma


# --- power method (Lemma lem:power) -----------------------------------------

def test_power_method_bracket_and_convergence():
    n = 256
    R, p, _ = _spd(n, 4)
    p1 = p.max()
    q = 3
    t = int(np.ceil(np.log(np.sqrt(4 * n))))
    lam, per = O.power_method(R, rng.power_start(n, q, 1), t)
    assert p1 / 6 <= lam <= p1 * (1 + 1e-14)
    assert np.all(per <= p1 * (1 + 1e-14))
    lam_long, _ = O.power_method(R, rng.power_start(n, 1, 1), 3000)
    assert abs(lam_long - p1) < 1e-9 * p1


def test_full_estimator_reaches_exact_entropy():
    R, p, _ = synth.dense_exp(128, 20.0, seed=4)
    H = O.entropy_of_spectrum(p)
    out = O.estimate(R, "chebyshev", m=30, s=400, seed=3, probe="gaussian")
    assert abs(out["H"] - H) / H < 0.03
    out = O.estimate(R, "taylor", m=60, s=400, seed=3, probe="gaussian", u_scale=1.0)
    assert abs(out["H"] - H) / H < 0.05


# --- planted mistakes ---------------------------------------------------------

def test_planted_mistakes_are_caught(monkeypatch):
    """Slips planted in the oracle make the spectral closed-form pins fail."""
    n, s, m = 24, 3, 6
    R, p, psi = _spd(n, 12)
    u = 1.1 * p.max()
    G = rng.gaussian(n, s, 2)
    proj2 = (psi.T @ G) ** 2
    ref_c = -(O.cheb_fm(p, u, m)[:, None] * proj2).sum() / s
    ref_t = np.log(1 / u) + sum(((p * (1 - p / u) ** k)[:, None] * proj2).sum() / k
                                for k in range(1, m + 1)) / s

    import oracle.vne_oracle as V
    good = V.cheb_coefficients

    def flipped(u_, m_):  # wrong sign on odd alpha_w
        a = good(u_, m_)
        a[3::2] *= -1
        return a

    monkeypatch.setattr(V, "cheb_coefficients", flipped)
    assert abs(V.chebyshev_estimate_clenshaw(R, G, u, m) - ref_c) > 1e-6
    monkeypatch.setattr(V, "cheb_coefficients", good)

    good_apply = V.apply_R
    monkeypatch.setattr(V, "apply_R", lambda R_, Y: good_apply(R_, Y) * (1 + 1e-3))
    assert abs(V.estimate(R, "taylor", m, s, 2, "gaussian", u=u)["H"] - ref_t) > 1e-7
    monkeypatch.setattr(V, "apply_R", good_apply)

    # a missing 1/k in the Taylor combine
    tau = V.taylor_terms(R, G, u, m)
    bad = np.log(1 / u) + tau[1:].sum() / s
    assert abs(bad - ref_t) > 1e-6
    assert abs(V.taylor_estimate_from_terms(tau, u) - ref_t) < 1e-12
