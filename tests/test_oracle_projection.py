"""Pins of the oracle's random-projection estimator (Algorithm alg:EN), CPU."""
import numpy as np
import pytest
from scipy import linalg

import oracle.projection as P
import synth
from oracle import rng


@pytest.mark.parametrize("n", [1, 2, 16, 64])
def test_hadamard_matches_library_and_is_orthogonal(n):
    H = P.hadamard(n)
    np.testing.assert_array_equal(H, linalg.hadamard(n) / np.sqrt(n))
    np.testing.assert_allclose(H.T @ H, np.eye(n), atol=1e-14)


def test_sketch_structure():
    n, s, seed = 64, 24, 9
    cs = P.sketch(n, s, "countsketch", seed)
    assert np.all((cs != 0).sum(axis=1) == 1)                 # one +-1 per row
    assert set(np.unique(cs[cs != 0])) <= {-1.0, 1.0}
    sr = P.sketch(n, s, "srht", seed)
    # every column is sqrt(n/s) * D h_i: norm sqrt(n/s), entries +-1/sqrt(s)
    np.testing.assert_allclose(np.linalg.norm(sr, axis=0), np.sqrt(n / s), rtol=1e-13)
    np.testing.assert_allclose(np.abs(sr), 1.0 / np.sqrt(s), rtol=1e-13)
    g = P.sketch(n, s, "gaussian", seed)
    np.testing.assert_allclose(g, rng.gaussian(n, s, seed) / np.sqrt(s))


@pytest.mark.parametrize("kind", ["gaussian", "srht", "countsketch"])
def test_sketch_isotropic_on_average(kind):
    n, s = 32, 64
    acc = np.zeros((n, n))
    T = 300
    for seed in range(T):
        Pi = P.sketch(n, s, kind, 1000 + seed)
        acc += Pi @ Pi.T
    acc /= T
    # E[Pi Pi^T] = I (CountSketch: s/s rows hit -> also I on the diagonal)
    np.testing.assert_allclose(np.diag(acc), 1.0, atol=0.15)
    off = acc - np.diag(np.diag(acc))
    assert np.abs(off).max() < 0.2


def test_orthogonal_sketch_recovers_spectrum_exactly():
    # with an orthogonal n x n "sketch" the singular values of R Pi are the
    # eigenvalues of R, so the estimate is the exact entropy of the top k
    n, k = 40, 7
    psi = synth.haar_orthogonal(n, 3)[:, :k]
    p = synth.spectrum_exponential(k, 2.0)
    R = (psi * p) @ psi.T
    Q = synth.haar_orthogonal(n, 5)
    sv = np.linalg.svd(R @ Q, compute_uv=False)[:k]
    np.testing.assert_allclose(np.sort(sv)[::-1], np.sort(p)[::-1], rtol=1e-12)
    H = float((p * np.log(1 / p)).sum())
    pos = sv[sv > 0]
    assert abs(float((pos * np.log(1 / pos)).sum()) - H) < 1e-12


@pytest.mark.parametrize("kind", ["gaussian", "srht", "countsketch"])
def test_low_rank_estimate_is_close(kind):
    # rank-10 density matrix, s = 256: the paper reports ~0.3 % errors
    n, k, s = 256, 10, 256
    psi = synth.haar_orthogonal(n, 11)[:, :k]
    p = synth.spectrum_exponential(k, 3.0)
    R = (psi * p) @ psi.T
    out = P.estimate_projection(R, k, s, kind, seed=4)
    H = float((p * np.log(1 / p)).sum())
    assert abs(out["H"] - H) / H < 0.1
    # Theorem thm:rp: |p_i^2 - p~_i^2| <= eps p_i^2 with a moderate eps here
    rel = np.abs(out["p"] ** 2 - p ** 2) / p ** 2
    assert rel.max() < 0.6


def test_srht_padding_equals_zero_padded_matrix():
    # n = 48 is read as R zero-padded to N = 64: R Pi equals the top n rows of
    # [R 0; 0 0] Pi_N, so the singular values agree
    n, N, k, s = 48, 64, 5, 32
    psi = synth.orthonormal_columns(n, k, 21)
    p = synth.spectrum_exponential(k, 2.0)
    R = synth.dense_density(psi, p)
    Rp = np.zeros((N, N))
    Rp[:n, :n] = R
    a = P.estimate_projection(R, k, s, "srht", seed=6)
    b = P.estimate_projection(Rp, k, s, "srht", seed=6)
    np.testing.assert_allclose(a["p"], b["p"], rtol=1e-12)
    assert abs(a["H"] - b["H"]) < 1e-12


def test_rank_deficient_tail_is_negligible():
    # rank 3 < k = 6: the trailing singular values are round-off
    n, s = 64, 16
    psi = synth.orthonormal_columns(n, 3, 2)
    p = np.array([0.5, 0.3, 0.2])
    R = synth.dense_density(psi, p)
    out = P.estimate_projection(R, 6, s, "gaussian", seed=3)
    assert np.all(out["p"][3:] < 1e-14)
    H = float((p * np.log(1 / p)).sum())
    assert abs(out["H"] - H) / H < 0.5


def test_rank_revealing_basis_is_orthonormal_on_the_kept_span():
    r = np.random.default_rng(0)
    V = r.standard_normal((60, 5)) @ r.standard_normal((5, 8))   # rank 5, 8 columns
    Q = P.rank_revealing_basis(V, np.linalg.eigvalsh(V.T @ V).max(), 1e-12)
    kept = np.linalg.norm(Q, axis=0) > 0.5
    assert kept.sum() == 5
    np.testing.assert_allclose(Q[:, kept].T @ Q[:, kept], np.eye(5), atol=1e-12)
    # same span as V
    proj = Q @ Q.T
    np.testing.assert_allclose(proj @ V, V, atol=1e-10)


def test_krylov_recovers_a_rank_k_spectrum_exactly():
    # the first block already spans range(R) (rank 6 <= b = 8): the Ritz
    # values are the eigenvalues, later blocks are round-off and dropped
    n, k = 120, 6
    psi = synth.orthonormal_columns(n, k, 5)
    p = synth.spectrum_exponential(k, 2.0)
    R = synth.dense_density(psi, p)
    out = P.estimate_block_krylov(R, k, 8, 3, "gaussian", seed=1)
    np.testing.assert_allclose(out["theta"], p, rtol=1e-11)
    H = float((p * np.log(1 / p)).sum())
    assert abs(out["H"] - H) < 1e-11          # tail: 1 - sum p = 0


def test_krylov_full_space_gives_exact_entropy():
    # q b >= n: K spans the whole space, T has R's spectrum, and the tail
    # formula is exact for a flat remainder
    n = 24
    R, p, _ = synth.dense_exp(n, 5.0, seed=3)
    theta = P.block_krylov_ritz(R, 8, 3, "gaussian", seed=2)
    np.testing.assert_allclose(theta, np.sort(p)[::-1], atol=1e-12)
    assert abs(P.krylov_entropy(theta, n, n) - float(-(p * np.log(p)).sum())) < 1e-12
    flat = np.full(30, 1 / 30)
    assert abs(P.krylov_entropy(flat[:10], 10, 30) - np.log(30)) < 1e-12


def test_krylov_ritz_values_interlace_from_below():
    # Ritz values never exceed the corresponding eigenvalues (Cauchy interlacing)
    n = 200
    R, p, _ = synth.dense_exp(n, 30.0, seed=4)
    theta = P.block_krylov_ritz(R, 8, 3, "srht", seed=3)
    ps = np.sort(p)[::-1]
    assert np.all(theta[:24] <= ps[:24] + 1e-14)
