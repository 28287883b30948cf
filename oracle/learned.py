"""CPU FP64 oracle of the learned moment correction (test infrastructure only;
only tests/, smoke() and the bench's CPU legs may use it).

The paper has no learned component: this is an extension of Algorithm 1b
(Section 3).  A low-degree Chebyshev estimate H_m = -(1/s) sum_k alpha_k
sum_j mu_{k,j} carries the truncation error of f_m (Lemma lem:prior); a small
network maps the first moments to that error so that m = 16 reaches the
accuracy of a much higher degree.

Contents (each written from its definition; "parity unpinned" nowhere: every
function has a pin in tests/test_oracle_learned.py):

* ``spectral_totals`` -- the per-degree probe totals sum_j mu_{k,j} of
  Algorithm 1b for R = Psi diag(p) Psi^T with Gaussian probes g_j = Psi z_j:
  g_j^T T_k(A) g_j = z_j^T T_k(diag) z_j = sum_i z_ij^2 T_k(x_i), with
  A = (2/u) R - I and x_i = 2 p_i / u - 1.  For Haar Psi and Gaussian g_j the
  z_j are again i.i.d. N(0, I), so the totals can be drawn from the spectrum
  alone, with z the Gaussian probe block of `seed` (counter j*n + i).
* ``features`` -- the 19 network inputs: tot_k / (s n) for k = 0..15,
  ln(n)/10, ln(lambda~)/10, ln(u)/10.
* ``target`` -- 100 (H(p) - H_16) / (n u), the correction the network
  learns.  With p_i = u y_i, h(p) - f_m(p) = u e_m(y) where e_m is the error
  of the degree-m Chebyshev truncation of y ln y on [0, 1] (the term y ln u is
  linear and expanded exactly), so H - H_m = -u sum_i e_m(y_i) + probe noise:
  divided by n u it is a mean over the spectral distribution of y, which the
  moment features tot_k / (s n) describe, whatever n is.
* the network: 19 -> 128 -> 128 -> 128 -> 1, GELU(x) = x Phi(x) (exact, erf)
  on the hidden layers, linear output; parameters are one flat vector
  [W1 (128x19 row-major), b1, W2 (128x128), b2, W3 (128x128), b3, W4 (1x128), b4];
  ``forward``, ``backward`` (chain rule written out, no autograd), the mean
  squared error and one Adam step (Kingma and Ba 2015).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from . import rng
from .vne_oracle import cheb_coefficients

N_IN, N_HID, N_OUT = 19, 128, 1
N_MOM = 16          # moments used as features (k = 0..15)
M_LOW = 16          # degree of the corrected estimator
LAYERS = [(N_IN, N_HID), (N_HID, N_HID), (N_HID, N_HID), (N_HID, N_OUT)]
N_PARAMS = sum(o * i + o for i, o in LAYERS)


def spectral_totals(p: np.ndarray, u: float, m: int, s: int, seed: int) -> np.ndarray:
    """sum_j mu_{k,j}, k = 0..m, for the spectrum p (see module docstring)."""
    p = np.asarray(p, dtype=np.float64)
    n = p.size
    z = rng.gaussian(n, s, seed)
    w = (z * z).sum(axis=1)
    x = 2.0 * p / u - 1.0
    T = np.polynomial.chebyshev.chebvander(x, m)  # T_k(x_i), k = 0..m
    return w @ T


def chebyshev_from_totals(tot: np.ndarray, u: float, s: int) -> float:
    """H_m = -(1/s) sum_k alpha_k tot_k (Algorithm 1b output)."""
    a = cheb_coefficients(u, tot.size - 1)
    return float(-(a * tot).sum() / s)


def features(tot: np.ndarray, s: int, n: int, lam: float, u: float) -> np.ndarray:
    f = np.empty(N_IN, dtype=np.float64)
    f[:N_MOM] = tot[:N_MOM] / (s * n)
    f[N_MOM] = np.log(n) / 10.0
    f[N_MOM + 1] = np.log(lam) / 10.0
    f[N_MOM + 2] = np.log(u) / 10.0
    return f


def entropy(p: np.ndarray) -> float:
    p = np.asarray(p, dtype=np.float64)
    q = p[p > 0]
    return float(-(q * np.log(q)).sum())


TARGET_SCALE = 100.0


def target(p: np.ndarray, H_low: float, u: float) -> float:
    return TARGET_SCALE * (entropy(p) - H_low) / (p.size * u)


# --------------------------------------------------------------------------
# the network
# --------------------------------------------------------------------------

def unpack(theta: np.ndarray):
    out, off = [], 0
    for i, o in LAYERS:
        W = theta[off:off + o * i].reshape(o, i)
        off += o * i
        b = theta[off:off + o]
        off += o
        out.append((W, b))
    return out


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def forward(theta: np.ndarray, X: np.ndarray):
    """Returns the output (B,) and the cache of pre-activations and inputs."""
    A = np.asarray(X, dtype=np.float64)
    cache = []
    layers = unpack(np.asarray(theta, dtype=np.float64))
    for li, (W, b) in enumerate(layers):
        Z = A @ W.T + b
        cache.append((A, Z))
        A = gelu(Z) if li + 1 < len(layers) else Z
    return A[:, 0], cache


def mse(y: np.ndarray, t: np.ndarray) -> float:
    return float(((y - t) ** 2).mean())


def backward(theta: np.ndarray, X: np.ndarray, t: np.ndarray):
    """Loss (mean squared error) and its gradient w.r.t. the flat parameters."""
    theta = np.asarray(theta, dtype=np.float64)
    y, cache = forward(theta, X)
    B = y.size
    dA = (2.0 / B) * (y - t)[:, None]
    layers = unpack(theta)
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        A_in, Z = cache[li]
        dZ = dA if li + 1 == len(layers) else dA * gelu_grad(Z)
        grads.append((dZ.T @ A_in, dZ.sum(axis=0)))
        dA = dZ @ W
    g = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in reversed(grads)])
    return mse(y, t), g


def adam_step(theta, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
