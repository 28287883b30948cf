"""CPU FP64 oracle of the random-projection estimator (test infrastructure
only; only tests/, smoke() and the bench's CPU legs may use it).

Algorithm alg:EN (Section 5): for R of rank at most k, sketch R~ = R Pi
(n x s) and return its (at most) k largest singular values p~_i and
H~ = sum_i p~_i ln(1/p~_i).  The random projection Pi is one of

* Gaussian: i.i.d. N(0, 1) entries (the experiments of Section 6), scaled
  by 1/sqrt(s) so that E[Pi Pi^T] = I (reading: the scaling is unstated);
* subsampled randomized Hadamard transform (Algorithm alg:SHD):
  Pi = D H S with D = diag(+-1), H the normalised N x N Hadamard matrix and
  S = s columns e_i drawn uniformly with replacement, scaled by sqrt(N/s) so
  that E[Pi Pi^T] = I (reading: Lemma lem:rp1 prints n/k where the usual
  normalisation is n/s).  H exists for N a power of two; for other n the
  matrix is read as R zero-padded to N = the next power of two, whose
  non-zero spectrum is that of R, so Pi is the first n rows of the N x s
  transform (reading: the paper assumes n a power of two);
* input-sparsity transform (Algorithm alg:IS): Pi = D S with each row of S a
  canonical row vector e_{h(j)}^T, h(j) uniform in {1..s}, unscaled.

Every random draw uses the SplitMix64 counter generator of ``oracle.rng``
(each side implements it separately):
  D_j      = Rademacher draw j of seed ^ 0xA0761D6478BD642F,
  Gaussian = the Gaussian probe block of seed, column t = probe t,
  i_t      = floor(u * n), u = (out(seed ^ 0xE7037ED1A0B428DB, t) >> 11) / 2^53,
  h(j)     = floor(u * s), u = (out(seed ^ 0xE7037ED1A0B428DB, j) >> 11) / 2^53.
"""
from __future__ import annotations

import numpy as np

from . import rng

D_SEED_XOR = 0xA0761D6478BD642F
IDX_SEED_XOR = 0xE7037ED1A0B428DB


def uniform_index(seed: int, count: int, m: int) -> np.ndarray:
    """floor(u * m) for the first `count` counters of the index stream."""
    out = rng.splitmix64(seed ^ IDX_SEED_XOR, np.arange(count, dtype=np.uint64))
    u = (out >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.minimum(np.floor(u * m).astype(np.int64), m - 1)


def signs(seed: int, n: int) -> np.ndarray:
    return rng.rademacher(n, 1, seed ^ D_SEED_XOR)[:, 0]


def hadamard(n: int) -> np.ndarray:
    """Normalised Sylvester Hadamard matrix, H_ij = (-1)^popcount(i & j) / sqrt(n)."""
    assert n > 0 and (n & (n - 1)) == 0, "n must be a power of two"
    i = np.arange(n)
    pc = np.vectorize(lambda v: bin(v).count("1"))(i[:, None] & i[None, :])
    return np.where(pc % 2 == 0, 1.0, -1.0) / np.sqrt(n)


def sketch(n: int, s: int, kind: str, seed: int) -> np.ndarray:
    """The random projection Pi (n x s, FP64) of Algorithm alg:EN."""
    if kind == "gaussian":
        return rng.gaussian(n, s, seed) / np.sqrt(s)
    if kind == "srht":
        N = 1 << max(0, (n - 1).bit_length())
        D = signs(seed, N)
        idx = uniform_index(seed, s, N)
        H = hadamard(N)
        S = np.zeros((N, s))
        S[idx, np.arange(s)] = 1.0
        return (np.sqrt(N / s) * (D[:, None] * (H @ S)))[:n]
    if kind == "countsketch":
        D = signs(seed, n)
        h = uniform_index(seed, n, s)
        Pi = np.zeros((n, s))
        Pi[np.arange(n), h] = D
        return Pi
    raise ValueError(kind)


def estimate_projection(R: np.ndarray, k: int, s: int, kind: str, seed: int) -> dict:
    """Algorithm alg:EN: singular values of R Pi, top k, and the entropy."""
    R = np.asarray(R, dtype=np.float64)
    n = R.shape[0]
    Pi = sketch(n, s, kind, seed)
    Rt = R @ Pi
    sv = np.linalg.svd(Rt, compute_uv=False)  # descending
    p = sv[:k]
    pos = p[p > 0]
    H = float((pos * np.log(1.0 / pos)).sum())
    return dict(H=H, p=p, sketch=Pi)


# --------------------------------------------------------------------------
# Block Krylov extension (not in the paper; the random-projection path of the
# batched workload: block b, q iterations, top-k Ritz values and a tail)
# --------------------------------------------------------------------------

def rank_revealing_basis(V: np.ndarray, lam_ref: float, drop: float) -> np.ndarray:
    """Orthonormal basis of the columns of V through the eigendecomposition
    of V^T V = U diag(l) U^T: Q = V U_kept diag(l_kept)^-1/2, keeping l_i >
    drop * lam_ref (lam_ref: the largest Gram eigenvalue of the first block,
    so directions at round-off level are dropped).  Dropped columns are zero."""
    l, U = np.linalg.eigh(V.T @ V)
    keep = l > drop * lam_ref
    M = np.zeros_like(U)
    M[:, keep] = U[:, keep] / np.sqrt(l[keep])
    return V @ M


def block_krylov_ritz(R: np.ndarray, b: int, q: int, kind: str, seed: int,
                      drop: float = 1e-12) -> np.ndarray:
    """Ritz values (descending) of R on K = span[Q_0 .. Q_{q-1}] with
    V_0 = R Pi, V_j = R Q_{j-1}, each V_j orthogonalised against the earlier
    blocks (two passes of block Gram-Schmidt) and then made orthonormal by
    rank_revealing_basis; T = K^T R K."""
    R = np.asarray(R, dtype=np.float64)
    n = R.shape[0]
    Pi = sketch(n, b, kind, seed)
    V = R @ Pi
    blocks, lam_ref = [], None
    for j in range(q):
        if j > 0:
            V = R @ blocks[-1]
            K = np.concatenate(blocks, axis=1)
            for _ in range(2):
                V = V - K @ (K.T @ V)
        if lam_ref is None:
            lam_ref = float(np.linalg.eigvalsh(V.T @ V).max())
        blocks.append(rank_revealing_basis(V, lam_ref, drop))
    K = np.concatenate(blocks, axis=1)
    T = K.T @ (R @ K)
    T = 0.5 * (T + T.T)
    return np.sort(np.linalg.eigvalsh(T))[::-1]


def krylov_entropy(theta: np.ndarray, k: int, n: int) -> float:
    """sum over the k largest Ritz values of t ln(1/t), plus the tail: the
    remaining trace 1 - sum_k theta_i spread evenly over the other n - k
    eigenvalues (reading of the tail estimate; tr R = 1)."""
    top = theta[:k]
    pos = top[top > 0]
    H = float((pos * np.log(1.0 / pos)).sum())
    rest = 1.0 - float(top.sum())
    if rest > 0 and n > k:
        H += rest * np.log((n - k) / rest)
    return H


def estimate_block_krylov(R, k: int, b: int, q: int, kind: str, seed: int,
                          drop: float = 1e-12) -> dict:
    theta = block_krylov_ritz(R, b, q, kind, seed, drop)
    return dict(H=krylov_entropy(theta, k, np.asarray(R).shape[0]), theta=theta[:k])
