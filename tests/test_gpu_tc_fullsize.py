"""Parity of the dense tensor-core path at the benchmark's launch shape, per probe.

The benchmark runs Algorithms 1a and 1b together on an n = 8192 density
matrix (p_i ~ i^-1.5 on the top n/4 states, a 1e-9 floor on the rest), with
s = 128 Gaussian probes and m = 40: every step is one launch over 2s = 256
probe columns (BN = 256, the K range split over CTA pairs, 64 k-blocks per
CTA).  These tests run that call at n = 1024, 4096 and 8192 with u from the
GPU's own power method, then evaluate the oracle at the same u:
  - the power method: u against the oracle's Algorithm alg:power;
  - every probe of a slice (the moments of each probe are independent of
    the others): each moment mu[k, j], tau[k, j], and the per-probe forms
    q_j = -sum_k alpha_k mu[k, j] (Algorithm 1b) and
    t_j = sum_{k>=1} tau[k, j] / k (Algorithm 1a);
  - the estimate over all 128 probes, at the GPU's own u (the FP64 path's u
    equals the oracle's to 1e-12 and is compared at the oracle's).
Tolerances (relative; moments relative to the largest entry of their row k):
  FP64     everything 1e-10.
  bf16x6   H 1e-6 (the split path's bar); per-probe forms and moments 1e-5:
           the FP32 master copy of Y bounds them (its rounding, ~6e-8, grows
           about linearly with the degree in the three-term recurrence).
  bf16x3   H 1e-5; forms 5e-5; moments 5e-4 (two pieces: products carry
           ~2^-16 relative error, and the accumulation into one FP32
           accumulator truncates; Taylor rows decay, so their relative error
           is larger).
  BF16     H 1e-3 (the mixed path's bar); per-probe forms 2e-2: one probe's
           form carries the bf16 rounding (2^-9) of R and Y without the
           averaging over probes that the estimate has.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle import rng

pytestmark = pytest.mark.gpu

vne = pytest.importorskip("paper_1801_01072_gb300")

M, S, SEED, T_POWER = 40, 128, 7, 30
SLICE = [0, 1, 2, 3, 60, 61, 126, 127]
TOL = {  # H, per-probe forms, moments
    "f64": (1e-10, 1e-10, 1e-10),
    "bf16x6": (1e-6, 1e-5, 1e-5),
    "bf16x3": (1e-5, 5e-5, 5e-4),
    "bf16": (1e-3, 2e-2, None),
}
U_TOL = {"f64": 1e-12, "bf16x6": 1e-6, "bf16x3": 1e-6, "bf16": 1e-4}


def rowerr(got, ref):
    sc = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-300)
    return float((np.abs(got - ref) / sc).max())


def forms(mu, tau, u):
    a = O.cheb_coefficients(u, mu.shape[0] - 1)
    k = np.arange(1, tau.shape[0], dtype=np.float64)
    return -(a[:, None] * mu).sum(axis=0), (tau[1:] / k[:, None]).sum(axis=0)


@pytest.fixture(scope="module", params=[1024, 4096, 8192])
def case(request):
    n = request.param
    R, p, _ = synth.dense_powerlaw(n, n // 4, 1.5, 1e-9, seed=2)
    lam, _ = O.power_method(R, rng.power_start(n, 1, SEED), T_POWER)
    G = rng.probes(n, S, SEED, "gaussian")
    return dict(n=n, R=R, Rd=torch.as_tensor(R).cuda(), lam=lam, G=G, oracle={})


def oracle_at(case, u):
    """The oracle's moments of all s probes at interval u (cached per u)."""
    if u not in case["oracle"]:
        case["oracle"][u] = (O.chebyshev_moments(case["R"], case["G"], u, M),
                             O.taylor_terms(case["R"], case["G"], u, M))
    return case["oracle"][u]


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "bf16x6", "f64"])
def test_fullsize_per_probe(case, prec):
    tol_H, tol_form, tol_mom = TOL[prec]
    b = vne.entropy_both(case["Rd"], M, S, seed=SEED, probe="gaussian", precision=prec,
                         power_iters=T_POWER, moments=True)
    # the interval: Algorithm alg:power on the same start vector
    u_ref = O.interval_u(case["lam"], 1.0)
    assert abs(b.u - u_ref) <= U_TOL[prec] * u_ref, (b.u, u_ref)
    # the device combine equals the combination of the device's own moments
    assert abs(b.H_chebyshev - O.chebyshev_estimate_from_moments(b.moments_chebyshev, b.u)) \
        <= 1e-12 * abs(b.H_chebyshev)
    assert abs(b.H_taylor - O.taylor_estimate_from_terms(b.moments_taylor, b.u)) \
        <= 1e-12 * abs(b.H_taylor)
    u = u_ref if prec == "f64" else b.u
    mu_all, tau_all = oracle_at(case, u)
    # per probe, on the slice
    mu, tau = mu_all[:, SLICE], tau_all[:, SLICE]
    gm, gt = b.moments_chebyshev[:, SLICE], b.moments_taylor[:, SLICE]
    if tol_mom is not None:
        assert rowerr(gm, mu) <= tol_mom, (prec, rowerr(gm, mu))
        assert rowerr(gt, tau) <= tol_mom, (prec, rowerr(gt, tau))
    qc, qt = forms(mu, tau, u)
    gc, gtt = forms(gm, gt, b.u)
    assert np.abs(gc - qc).max() <= tol_form * np.abs(qc).max(), (prec, np.abs(gc - qc).max())
    assert np.abs(gtt - qt).max() <= tol_form * np.abs(qt).max(), (prec, np.abs(gtt - qt).max())
    # the estimate over all s probes
    Hc = O.chebyshev_estimate_from_moments(mu_all, u)
    Ht = O.taylor_estimate_from_terms(tau_all, u)
    assert abs(b.H_chebyshev - Hc) <= tol_H * abs(Hc), (prec, b.H_chebyshev, Hc)
    assert abs(b.H_taylor - Ht) <= tol_H * abs(Ht), (prec, b.H_taylor, Ht)
