"""Seeded synthetic density matrices shaped like the paper's workloads.

This module only builds inputs.  It holds none of the estimators'
arithmetic (no entropy, no polynomial, no trace estimate, no power
method): both the CUDA path's tests and the CPU oracle draw their
matrices from here, and nothing else is shared between them.

Input model (Section 1.1, eqs. R and R1): a real density matrix is
R = Psi diag(p) Psi^T with orthonormal columns psi_i, p_i > 0 and
sum p_i = 1.  The paper draws its dense matrices from QETLAB's
RandomDensityMatrix (Section 6), which is not available here; Haar-like
orthonormal Psi from the QR factorisation of a seeded Gaussian matrix
stands in for it.  The banded matrices follow the paper's tridiagonal
Poisson example (Section 6, eq. poisson_matrix) and its wider,
diagonally dominant generalisation.

Banded storage (DIA, symmetric): ``vals[d, i] = R[i, i + d]`` for
d = 0 .. D-1 and i < n - d; entries with i >= n - d are zero padding.
The lower triangle is implied by symmetry.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "spectrum_exponential",
    "spectrum_powerlaw_floor",
    "spectrum_poisson",
    "haar_orthogonal",
    "dense_density",
    "dense_exp",
    "dense_powerlaw",
    "orthonormal_columns",
    "dense_lowrank",
    "hermitian_density",
    "batched_specs",
    "training_spectrum",
    "learned_sample_params",
    "mlp_init",
    "band_diag_dominant",
    "band_poisson",
    "dia_to_dense",
    "WORKLOADS",
]


def spectrum_exponential(n: int, tau: float) -> np.ndarray:
    """p_i proportional to exp(-i/tau), i = 1..n, normalised to unit sum."""
    i = np.arange(1, n + 1, dtype=np.float64)
    p = np.exp(-i / tau)
    return p / p.sum()


def spectrum_powerlaw_floor(n: int, k: int, alpha: float, floor: float) -> np.ndarray:
    """p_i proportional to i^-alpha for i <= k, a constant floor for i > k,
    then renormalised to unit sum (the floor is applied before scaling)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    p = np.where(i <= k, i ** (-alpha), 0.0)
    p = p / p.sum()
    p = np.where(i <= k, p, floor)
    return p / p.sum()


def spectrum_poisson(n: int) -> np.ndarray:
    """Eigenvalues of tridiag(-1, 2, -1) / (2n), eq. trig_eigs of Section 6:
    lambda_i = (4 / 2n) sin^2(i pi / (2n + 2)), i = 1..n (ascending)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return (4.0 / (2.0 * n)) * np.sin(i * np.pi / (2.0 * n + 2.0)) ** 2


def haar_orthogonal(n: int, seed: int) -> np.ndarray:
    """Q of the QR factorisation of a seeded n x n N(0,1) matrix (FP64)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n))
    q, r = np.linalg.qr(a)
    # sign fix so that Q is Haar distributed (the diagonal of r made positive)
    q *= np.sign(np.diag(r))[None, :]
    return q


def dense_density(psi: np.ndarray, p: np.ndarray) -> np.ndarray:
    """R = Psi diag(p) Psi^T, symmetrised, row-major FP64 (eq. R1)."""
    r = (psi * p[None, :]) @ psi.T
    r = 0.5 * (r + r.T)
    return np.ascontiguousarray(r)


def dense_exp(n: int = 512, tau: float = 50.0, seed: int = 1):
    """Dense density matrix with p_i ~ exp(-i/tau); returns (R, p, Psi)."""
    psi = haar_orthogonal(n, seed)
    p = spectrum_exponential(n, tau)
    return dense_density(psi, p), p, psi


def dense_powerlaw(n: int = 8192, k: int = 2048, alpha: float = 1.5,
                   floor: float = 1e-9, seed: int = 2):
    """Dense density matrix with p_i ~ i^-alpha on the top k states and a
    floor on the rest; returns (R, p, Psi)."""
    psi = haar_orthogonal(n, seed)
    p = spectrum_powerlaw_floor(n, k, alpha, floor)
    return dense_density(psi, p), p, psi


def orthonormal_columns(n: int, k: int, seed: int) -> np.ndarray:
    """n x k with orthonormal columns: Q of the QR factorisation of a seeded
    n x k N(0,1) matrix, sign-fixed (the first k columns of a Haar matrix)."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((n, k)))
    return q * np.sign(np.diag(r))[None, :]


def dense_lowrank(n: int = 8192, k: int = 64, tau: float = 16.0, seed: int = 4):
    """Density matrix of rank k (a mixture of k pure states, the setting of
    Algorithm alg:EN) with p_i ~ exp(-i/tau); returns (R, p, Psi)."""
    psi = orthonormal_columns(n, k, seed)
    p = spectrum_exponential(k, tau)
    return dense_density(psi, p), p, psi


def hermitian_density(n: int, p: np.ndarray, seed: int) -> np.ndarray:
    """Complex Hermitian density matrix R = U diag(p) U^H, U the sign-fixed Q of
    a seeded complex Ginibre matrix (Haar unitary); complex128, row-major."""
    r = np.random.default_rng(seed)
    a = (r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))) / np.sqrt(2.0)
    q, rr = np.linalg.qr(a)
    d = np.diag(rr)
    q = q * (d / np.abs(d))[None, :]
    R = (q * np.asarray(p, dtype=np.float64)[None, :]) @ q.conj().T
    return np.ascontiguousarray(0.5 * (R + R.conj().T))


def batched_specs(count: int, seed: int, n_lo: int = 256, n_hi: int = 4096):
    """Sizes and spectra of a batch of uneven dense density matrices: n
    log-uniform in [n_lo, n_hi], p_i ~ exp(-i/tau) with tau ~ U(10, n/4), and a
    seed for each matrix's Haar eigenvectors.  Returns a list of (n, p, seed)."""
    r = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(np.exp(r.uniform(np.log(n_lo), np.log(n_hi))))
        tau = r.uniform(10.0, n / 4.0)
        out.append((n, spectrum_exponential(n, tau), int(r.integers(1, 2 ** 31))))
    return out


def training_spectrum(kind: int, n: int, a: float, ktop: int, floor: float) -> np.ndarray:
    """Spectra of the learned correction's training set, unit trace, i = 1..n:
    kind 0: p_i ~ exp(-(i-1)/a); kind 1: p_i ~ i^-a for i <= ktop, floor beyond."""
    i = np.arange(1, n + 1, dtype=np.float64)
    if kind == 0:
        q = np.exp(-(i - 1.0) / a)
    else:
        q = np.where(i <= ktop, i ** -a, floor)
    return q / q.sum()


def learned_sample_params(count: int, seed: int, n_lo: int = 1024, n_hi: int = 4096) -> dict:
    """Seeded parameters of `count` training spectra: half exponential with
    a = tau ~ U(10, n/4), half power law with a = alpha ~ U(1.1, 2.0),
    ktop ~ U(n/8, n/2) and a floor log-uniform in [1e-10, 1e-6]; n
    log-uniform in [n_lo, n_hi]; u = c * p_1 with c ~ U(1.0, 1.1); one probe
    seed per spectrum.  Arrays are int32 / float32 / uint64."""
    r = np.random.default_rng(seed)
    n = np.exp(r.uniform(np.log(n_lo), np.log(n_hi), count)).astype(np.int32)
    kind = (np.arange(count) % 2).astype(np.int32)
    tau = r.uniform(10.0, n / 4.0)
    alpha = r.uniform(1.1, 2.0, count)
    a = np.where(kind == 0, tau, alpha).astype(np.float32)
    ktop = r.uniform(n / 8.0, n / 2.0).astype(np.int32)
    floor = np.exp(r.uniform(np.log(1e-10), np.log(1e-6), count)).astype(np.float32)
    c = r.uniform(1.0, 1.1, count).astype(np.float32)
    seeds = r.integers(1, 2 ** 62, count, dtype=np.int64).astype(np.uint64)
    return dict(kind=kind, n=n, a=a, ktop=ktop, floor=floor, c=c, seed=seeds)


def mlp_init(seed: int, layers=((19, 128), (128, 128), (128, 128), (128, 1))) -> np.ndarray:
    """Initial parameters of the correction network, one flat vector
    [W1 (out x in, row-major), b1, W2, b2, ...]: U(-1/sqrt(in), 1/sqrt(in))."""
    r = np.random.default_rng(seed)
    parts = []
    for i, o in layers:
        lim = 1.0 / np.sqrt(i)
        parts.append(r.uniform(-lim, lim, o * i))
        parts.append(r.uniform(-lim, lim, o))
    return np.concatenate(parts)


def band_diag_dominant(n: int, half_bw: int = 16, offdiag_scale: float = 0.02,
                       seed: int = 3, dtype=np.float32) -> np.ndarray:
    """Symmetric banded density matrix in DIA storage, shape (half_bw+1, n).

    Off-diagonals are U(-1, 1) * offdiag_scale, the diagonal is
    1 + sum_j |R_ij| over the row's off-diagonal entries (strict diagonal
    dominance, so R is SPD), and the whole matrix is divided by its trace.
    """
    rng = np.random.default_rng(seed)
    D = half_bw + 1
    vals = np.zeros((D, n), dtype=np.float64)
    rowabs = np.zeros(n, dtype=np.float64)
    for d in range(1, D):
        v = rng.uniform(-1.0, 1.0, n - d) * offdiag_scale
        vals[d, : n - d] = v
        a = np.abs(v)
        rowabs[: n - d] += a   # row i holds R[i, i+d]
        rowabs[d:] += a        # row i+d holds R[i+d, i]
    vals[0] = 1.0 + rowabs
    vals /= vals[0].sum()
    return np.ascontiguousarray(vals.astype(dtype))


def band_poisson(n: int, dtype=np.float64) -> np.ndarray:
    """tridiag(-1, 2, -1) / (2n) in DIA storage, shape (2, n) (Section 6)."""
    vals = np.zeros((2, n), dtype=np.float64)
    vals[0] = 2.0
    vals[1, : n - 1] = -1.0
    vals /= 2.0 * n
    return np.ascontiguousarray(vals.astype(dtype))


def dia_to_dense(vals: np.ndarray) -> np.ndarray:
    """Expand symmetric DIA storage to a dense FP64 matrix (small n only)."""
    D, n = vals.shape
    r = np.zeros((n, n), dtype=np.float64)
    v = vals.astype(np.float64)
    r[np.arange(n), np.arange(n)] = v[0]
    for d in range(1, D):
        idx = np.arange(n - d)
        r[idx, idx + d] = v[d, : n - d]
        r[idx + d, idx] = v[d, : n - d]
    return r


# Named workloads: (what it is, sizes).  The estimator parameters sit
# beside the matrix recipe so that tests and the bench use one definition.
WORKLOADS = {
    "dense_exp_n512": dict(kind="dense", n=512, spectrum="exp", tau=50.0, seed=1,
                           m=20, s=50, probe="rademacher", power_iters=30),
    "dense_powerlaw_n8192": dict(kind="dense", n=8192, spectrum="powerlaw", k=2048,
                                 alpha=1.5, floor=1e-9, seed=2, m=40, s=128,
                                 probe="gaussian", power_iters=30),
    "band33_n1e7": dict(kind="band", n=10_000_000, half_bw=16, offdiag_scale=0.02,
                        seed=3, m=30, s=64, probe="rademacher", power_iters=30),
    # the dense n = 8192 matrix through the degree-16 estimator plus the learned
    # correction (trained on 100k sampled spectra, n = 1024..4096), against
    # the plain degree-64 estimator
    "learned_n8192": dict(kind="learned", n=8192, spectrum="powerlaw", k=2048, alpha=1.5,
                          floor=1e-9, seed=2, m=16, s=128, probe="gaussian", power_iters=30,
                          train_count=100000, train_epochs=20, m_ref=64),
    # a random 5000 x 5000 complex density matrix (Section 6, Hermitian case):
    # Haar eigenvectors, p_i ~ exp(-i/500); Taylor m = 10 and Chebyshev m = 10,
    # s = 100 real Gaussian probes, u from the power method
    "hermitian_n5000": dict(kind="hermitian", n=5000, tau=500.0, seed=6, m=10, s=100,
                            probe="gaussian"),
    # 256 uneven dense matrices in one batched call (one CUDA graph launch)
    "batched256": dict(kind="batched", count=256, n_lo=256, n_hi=4096, seed=5, m=24, s=32,
                       probe="gaussian", power_iters=30),
    # rank-64 mixture for the random-projection estimator (Algorithm alg:EN)
    "lowrank_n8192_k64": dict(kind="lowrank", n=8192, k=64, tau=16.0, seed=4, s=256,
                              sketch="gaussian"),
    # the same matrix through the block-Krylov extension: block 64, 4 iterations,
    # top-64 Ritz values and the tail
    "krylov_n8192_b64": dict(kind="lowrank", n=8192, k=64, tau=16.0, seed=4, s=64,
                             sketch="gaussian", krylov=4),
    # the same band at n = 2e6 (profiling captures of the banded kernels)
    "band33_n2e6": dict(kind="band", n=2_000_000, half_bw=16, offdiag_scale=0.02,
                        seed=3, m=30, s=64, probe="rademacher", power_iters=30),
}
