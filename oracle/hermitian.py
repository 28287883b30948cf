"""CPU FP64 oracle of the Hermitian estimators (test infrastructure only;
only tests/, smoke() and the bench's CPU legs may use it).

Section 4 (Approaches for Hermitian Density Matrices): a complex Hermitian
PSD R = B + iC has a real symmetric PSD part B (Theorem thm:hermitian1) and
tr R = tr B (Theorem thm:hermitian2).  Algorithms alg1a_complex and
alg1b_complex keep real Gaussian probes g_j and return

  Taylor:     (1/s) sum_j sum_{k=1..m} g_j^T Re[R (I - R)^k] g_j / k,
  Chebyshev: -(1/s) sum_j g_j^T Re[f_m(R)] g_j,

with one as the upper bound of the spectrum in place of u.  This module
evaluates them in complex arithmetic, as printed: the matrix powers act on
complex blocks and only the final quadratic forms take the real part.  The
general u of Algorithms 1a/1b is kept as a parameter (reading: u = 1 is the
printed choice and the default; the Taylor constant is then ln(1/u) = 0).
"""
from __future__ import annotations

import numpy as np

from .vne_oracle import cheb_coefficients


def chebyshev_moments_complex(R: np.ndarray, G: np.ndarray, u: float, m: int) -> np.ndarray:
    """mu[k, j] = g_j^T Re[T_k((2/u) R - I)] g_j, k = 0..m (three-term
    recurrence on complex blocks Y_k = T_k((2/u) R - I) G)."""
    R = np.asarray(R, dtype=np.complex128)
    G = np.asarray(G, dtype=np.float64)
    mu = np.zeros((m + 1, G.shape[1]))
    mu[0] = (G * G).sum(axis=0)
    if m == 0:
        return mu
    y_prev = G.astype(np.complex128)
    y = (2.0 / u) * (R @ y_prev) - y_prev
    mu[1] = (G * y.real).sum(axis=0)
    for k in range(2, m + 1):
        y_next = 2.0 * ((2.0 / u) * (R @ y) - y) - y_prev
        y_prev, y = y, y_next
        mu[k] = (G * y.real).sum(axis=0)
    return mu


def chebyshev_estimate_complex(R, G, u: float, m: int) -> float:
    a = cheb_coefficients(u, m)
    mu = chebyshev_moments_complex(R, G, u, m)
    return float(-(a[:, None] * mu).sum() / G.shape[1])


def taylor_terms_complex(R: np.ndarray, G: np.ndarray, u: float, m: int) -> np.ndarray:
    """tau[k, j] = g_j^T Re[R (I - R/u)^k] g_j, k = 0..m."""
    R = np.asarray(R, dtype=np.complex128)
    G = np.asarray(G, dtype=np.float64)
    tau = np.zeros((m + 1, G.shape[1]))
    y = G.astype(np.complex128)              # (I - R/u)^k g
    for k in range(m + 1):
        z = R @ y
        tau[k] = (G * z.real).sum(axis=0)
        y = y - z / u
    return tau


def taylor_estimate_complex(R, G, u: float, m: int) -> float:
    tau = taylor_terms_complex(R, G, u, m)
    k = np.arange(1, m + 1)
    return float(np.log(1.0 / u) + (tau[1:] / k[:, None]).sum() / G.shape[1])
