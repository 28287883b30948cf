"""Plain, slow CPU FP64 oracle for the randomized von Neumann entropy
estimators of Kontopoulou, Dexter, Szpankowski, Grama and Drineas,
"Randomized linear algebra approaches to estimate the von Neumann entropy
of density matrices" (arXiv:1801.01072).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline legs of ``bench.py`` may import, call or execute
anything under ``oracle/``.  The CUDA library never routes through it and
shares no code with it; the only common module is ``synth`` (seeded input
matrices, none of the method's arithmetic).

Every function computes in FP64 with NumPy, in the paper's order and
notation, and names the passage it follows.  Library primitives (matrix
products, ``eigh``) serve as single steps; there is no blocking or
fusion.  Where the paper is silent or ambiguous the reading taken is
stated at the function.

Operators: ``R`` is either a dense (n, n) array or a :class:`Dia`
(symmetric banded storage ``vals[d, i] = R[i, i + d]``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import rng

# --------------------------------------------------------------------------
# Operators
# --------------------------------------------------------------------------


@dataclass
class Dia:
    """Symmetric banded matrix: vals[d, i] = R[i, i+d], d = 0..D-1."""

    vals: np.ndarray  # (D, n), any float dtype; used in FP64

    @property
    def n(self) -> int:
        return self.vals.shape[1]


def size_of(R) -> int:
    return R.n if isinstance(R, Dia) else R.shape[0]


def apply_R(R, Y: np.ndarray) -> np.ndarray:
    """R @ Y for a dense or symmetric-banded R (FP64).

    For banded R the product is written out by diagonals:
    (RY)_i = sum_d R[i,i+d] Y_{i+d} + sum_{d>0} R[i-d,i] Y_{i-d}.
    """
    Y = np.asarray(Y, dtype=np.float64)
    if not isinstance(R, Dia):
        return np.asarray(R, dtype=np.float64) @ Y
    v = R.vals.astype(np.float64)
    D, n = v.shape
    col = Y.ndim == 1
    Y2 = Y[:, None] if col else Y
    Z = v[0][:, None] * Y2
    for d in range(1, D):
        if d >= n:
            break
        a = v[d, : n - d][:, None]
        Z[: n - d] += a * Y2[d:]
        Z[d:] += a * Y2[: n - d]
    return Z[:, 0] if col else Z


def trace_of(R) -> float:
    if isinstance(R, Dia):
        return float(R.vals[0].astype(np.float64).sum())
    return float(np.trace(np.asarray(R, dtype=np.float64)))


# --------------------------------------------------------------------------
# Exact entropy (eqs. earlyR and VN, Section 1.1)
# --------------------------------------------------------------------------


def entropy_of_spectrum(p: np.ndarray) -> float:
    """H = -sum_{p_i > 0} p_i ln p_i; p_i ln p_i := 0 for p_i = 0 (footnote
    to eq. earlyR).  Non-positive eigenvalues (round-off) count as zero."""
    p = np.asarray(p, dtype=np.float64)
    q = p[p > 0]
    return float(-(q * np.log(q)).sum())


def exact_entropy(R) -> float:
    """Exact H(R) from a full symmetric eigendecomposition (eq. VN)."""
    if isinstance(R, Dia):
        from synth import dia_to_dense  # input-model expansion only

        R = dia_to_dense(R.vals)
    w = np.linalg.eigvalsh(np.asarray(R, dtype=np.float64))
    return entropy_of_spectrum(w)


# --------------------------------------------------------------------------
# Power method (Appendix, Algorithm alg:power; Lemma lem:power)
# --------------------------------------------------------------------------


def power_method(R, X0: np.ndarray, t: int):
    """Algorithm alg:power on q start vectors (columns of X0).

    x_i = R x_{i-1} for i = 1..t, then p1^j = x_t^T R x_t / x_t^T x_t and
    p1 = max_j p1^j.  Reading: each iterate is divided by its 2-norm.  The
    printed algorithm does not normalise, which over- or underflows for
    t in the tens (R has unit trace, so ||R^t x|| shrinks like p_1^t); the
    Rayleigh quotient is unchanged by the scaling in exact arithmetic.
    Returns (p1, per-trial values).
    """
    X = np.array(X0, dtype=np.float64, copy=True)
    if X.ndim == 1:
        X = X[:, None]
    X /= np.linalg.norm(X, axis=0)[None, :]
    for _ in range(t):
        X = apply_R(R, X)
        X /= np.linalg.norm(X, axis=0)[None, :]
    RX = apply_R(R, X)
    per = (X * RX).sum(axis=0) / (X * X).sum(axis=0)
    return float(per.max()), per


def interval_u(p1: float, u_scale: float = 1.0) -> float:
    """u = min{1, c * p1} (Algorithms 1a/1b step 3 print c = 6; the
    experiments of Section 6 use c = 1 and c = 6; c is a parameter)."""
    return float(min(1.0, u_scale * p1))


# --------------------------------------------------------------------------
# Chebyshev expansion of h(x) = x ln x on [0, u] (Section 3, Lemma lem:prior)
# --------------------------------------------------------------------------


def cheb_coefficients(u: float, m: int) -> np.ndarray:
    """alpha_0 = (u/2)(ln(u/4) + 1), alpha_1 = (u/4)(2 ln(u/4) + 3),
    alpha_w = (-1)^w u / (w^3 - w) for w >= 2 (Lemma lem:prior)."""
    a = np.zeros(m + 1, dtype=np.float64)
    a[0] = (u / 2.0) * (np.log(u / 4.0) + 1.0)
    if m >= 1:
        a[1] = (u / 4.0) * (2.0 * np.log(u / 4.0) + 3.0)
    for w in range(2, m + 1):
        a[w] = (-1.0) ** w * u / (w ** 3 - w)
    return a


def cheb_T(w: int, x, u: float):
    """T_w on [0, u]: cos(w arccos((2/u) x - 1)) (Section 3).  Outside
    [0, u] the same polynomial is continued by cosh(w arccosh t)."""
    t = (2.0 / u) * np.asarray(x, dtype=np.float64) - 1.0
    out = np.empty_like(t)
    inside = np.abs(t) <= 1.0
    out[inside] = np.cos(w * np.arccos(t[inside]))
    hi = t > 1.0
    out[hi] = np.cosh(w * np.arccosh(t[hi]))
    lo = t < -1.0
    out[lo] = (-1.0) ** w * np.cosh(w * np.arccosh(-t[lo]))
    return out


def cheb_fm(x, u: float, m: int):
    """f_m(x) = sum_{w=0}^m alpha_w T_w(x) (Section 3, Lemma lem:prior)."""
    a = cheb_coefficients(u, m)
    x = np.asarray(x, dtype=np.float64)
    return sum(a[w] * cheb_T(w, x, u) for w in range(m + 1))


# --------------------------------------------------------------------------
# NTE: exact polynomial traces, no trace estimation (Section 6)
# --------------------------------------------------------------------------


def nte_chebyshev(p: np.ndarray, u: float, m: int) -> float:
    """-tr f_m(R) = -sum_i f_m(p_i) (eq. cheb_no_trace)."""
    return float(-cheb_fm(np.asarray(p, dtype=np.float64), u, m).sum())


def nte_taylor(p: np.ndarray, u: float, m: int) -> float:
    """ln u^-1 + sum_{k=1}^m tr(R (I - R/u)^k) / k with tr taken over the
    spectrum (Lemma lem1a truncated at m terms)."""
    p = np.asarray(p, dtype=np.float64)
    tot = np.log(1.0 / u)
    for k in range(1, m + 1):
        tot += (p * (1.0 - p / u) ** k).sum() / k
    return float(tot)


# --------------------------------------------------------------------------
# Algorithm 1b (Chebyshev) with the Clenshaw evaluation of Appendix C
# --------------------------------------------------------------------------


def clenshaw_quadforms(R, G: np.ndarray, u: float, m: int) -> np.ndarray:
    """g_j^T f_m(R) g_j for every column g_j of G (Algorithm alg_clenshaw_mv).

    y_{m+2} = y_{m+1} = 0; for k = m..0:
    y_k = alpha_k g + (4/u) R y_{k+1} - 2 y_{k+1} - y_{k+2};
    result = (alpha_0 g^T g + g^T (y_0 - y_2)) / 2.
    """
    G = np.asarray(G, dtype=np.float64)
    a = cheb_coefficients(u, m)
    y1 = np.zeros_like(G)  # y_{k+1}
    y2 = np.zeros_like(G)  # y_{k+2}
    ys = {}
    for k in range(m, -1, -1):
        yk = a[k] * G + (4.0 / u) * apply_R(R, y1) - 2.0 * y1 - y2
        if k <= 2:
            ys[k] = yk
        y2, y1 = y1, yk
    y_2 = ys[2] if m >= 2 else np.zeros_like(G)
    gg = (G * G).sum(axis=0)
    return 0.5 * (a[0] * gg + (G * (ys[0] - y_2)).sum(axis=0))


def chebyshev_estimate_clenshaw(R, G: np.ndarray, u: float, m: int) -> float:
    """Algorithm 1b output: -(1/s) sum_j g_j^T f_m(R) g_j."""
    return float(-clenshaw_quadforms(R, G, u, m).mean())


# --------------------------------------------------------------------------
# Forward three-term recurrence with per-probe moments (second formulation)
# --------------------------------------------------------------------------


def chebyshev_moments(R, G: np.ndarray, u: float, m: int) -> np.ndarray:
    """mu[k, j] = g_j^T T_k(R) g_j, k = 0..m, by the forward recurrence of
    the Chebyshev polynomials in the mapped matrix (2/u) R - I:
    Y_0 = G, Y_1 = (2/u) R G - G, Y_k = 2((2/u) R - I) Y_{k-1} - Y_{k-2}.
    Then g^T f_m(R) g = sum_k alpha_k mu_k (Section 3 definition of f_m)."""
    G = np.asarray(G, dtype=np.float64)
    mu = np.zeros((m + 1, G.shape[1]), dtype=np.float64)
    mu[0] = (G * G).sum(axis=0)
    if m == 0:
        return mu
    y_prev = G
    y = (2.0 / u) * apply_R(R, G) - G
    mu[1] = (G * y).sum(axis=0)
    for k in range(2, m + 1):
        y_next = 2.0 * ((2.0 / u) * apply_R(R, y) - y) - y_prev
        y_prev, y = y, y_next
        mu[k] = (G * y).sum(axis=0)
    return mu


def chebyshev_estimate_from_moments(mu: np.ndarray, u: float) -> float:
    """-(1/s) sum_j sum_k alpha_k mu[k, j] (Algorithm 1b output)."""
    m = mu.shape[0] - 1
    a = cheb_coefficients(u, m)
    return float(-(a[:, None] * mu).sum() / mu.shape[1])


# --------------------------------------------------------------------------
# Algorithm 1a (Taylor)
# --------------------------------------------------------------------------


def taylor_terms(R, G: np.ndarray, u: float, m: int) -> np.ndarray:
    """tau[k, j] = g_j^T R (I - R/u)^k g_j for k = 0..m (Algorithm 1a).

    C^k g is built by y_k = y_{k-1} - (1/u) R y_{k-1} from y_0 = g and
    contracted with w = R g: tau_k = w^T y_k.  (Rewriting the term as
    u (g^T C^k g - g^T C^{k+1} g) is avoided: it cancels.)"""
    G = np.asarray(G, dtype=np.float64)
    W = apply_R(R, G)
    tau = np.zeros((m + 1, G.shape[1]), dtype=np.float64)
    y = G
    tau[0] = (W * y).sum(axis=0)
    for k in range(1, m + 1):
        y = y - (1.0 / u) * apply_R(R, y)
        tau[k] = (W * y).sum(axis=0)
    return tau


def taylor_estimate_from_terms(tau: np.ndarray, u: float) -> float:
    """ln u^-1 + (1/s) sum_j sum_{k=1}^m tau[k, j] / k (Algorithm 1a)."""
    m = tau.shape[0] - 1
    k = np.arange(1, m + 1, dtype=np.float64)
    return float(np.log(1.0 / u) + (tau[1:] / k[:, None]).sum() / tau.shape[1])


# --------------------------------------------------------------------------
# Whole estimators (power method -> u -> probes -> recurrence -> combine)
# --------------------------------------------------------------------------


def estimate(R, method: str, m: int, s: int, seed: int, probe: str = "rademacher",
             power_iters: int = 30, power_trials: int = 1, u_scale: float = 1.0,
             u: float | None = None, probe_cols=None) -> dict:
    """Algorithm 1a (method="taylor") or 1b (method="chebyshev").

    If ``u`` is given the power method is skipped.  ``probe_cols`` limits
    the evaluation to a subset of the s probes (their moments are exact
    per probe; the returned H is then over that subset only).
    """
    n = size_of(R)
    lam = None
    if u is None:
        X0 = rng.power_start(n, power_trials, seed)
        lam, _ = power_method(R, X0, power_iters)
        u = interval_u(lam, u_scale)
    G = rng.probes(n, s, seed, probe)
    if probe_cols is not None:
        G = G[:, probe_cols]
    if method == "chebyshev":
        mom = chebyshev_moments(R, G, u, m)
        H = chebyshev_estimate_from_moments(mom, u)
    elif method == "taylor":
        mom = taylor_terms(R, G, u, m)
        H = taylor_estimate_from_terms(mom, u)
    else:
        raise ValueError(method)
    return dict(H=H, u=u, lam=lam, moments=mom)


def suggest_m(method: str, u: float, ell: float, eps: float) -> int:
    """m of Theorem thm:taylor (ceil((u/ell) ln(1/eps))) or Theorem
    thm:cheb (sqrt(u / (2 eps ell ln(1/(1-ell)))), rounded up)."""
    if method == "taylor":
        return int(np.ceil((u / ell) * np.log(1.0 / eps)))
    return int(np.ceil(np.sqrt(u / (2.0 * eps * ell * np.log(1.0 / (1.0 - ell))))))
