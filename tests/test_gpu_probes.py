"""Estimators on probes the caller gives (vne_entropy_chebyshev_probes /
vne_entropy_taylor_probes, through the C ABI).

Checks:
  - the seed's own Rademacher probes, passed in, reproduce the seeded call
    bit for bit (dense FP64 and BF16: the same kernels see the same values);
  - a probe along an eigenvector psi_1 of R = Psi diag(p) Psi^T gives the
    closed forms psi_1^T f_m(R) psi_1 = f_m(p_1) (Section 3) and
    sum_k psi_1^T R (I - R/u)^k psi_1 / k = sum_k p_1 (1 - p_1/u)^k / k
    (Section 2), in FP64 and in bf16x6 (one probe carries the per-moment
    rounding of the FP32 master without averaging: 1e-5, the split modes'
    moment tolerance);
  - unit-vector probes e_i against the oracle's quadratic forms, element by
    element; a zero probe gives zero moments;
  - Gaussian probes on the banded FP32 path (the bulk-copy kernel, S = 32)
    against the oracle, at the FP32 banded tolerance 2e-5.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle import rng

pytestmark = pytest.mark.gpu

vne = pytest.importorskip("paper_1801_01072_gb300")


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype).cuda()


@pytest.mark.parametrize("precision", ["f64", "bf16"])
def test_seeded_probes_passed_in_are_bit_identical(precision):
    n, m, s, seed = 300, 10, 24, 5
    R, p, _ = synth.dense_exp(n, 30.0, seed=2)
    u = 1.02 * p.max()
    G = rng.probes(n, s, seed, "rademacher")
    gt = torch.float64 if precision == "f64" else torch.float32
    for method, fn in (("chebyshev", vne.entropy_chebyshev), ("taylor", vne.entropy_taylor)):
        a = fn(dev(R), m, s, seed=seed, u=u, precision=precision, moments=True)
        b = vne.entropy_with_probes(dev(R), dev(G, gt), m, method=method, u=u,
                                    precision=precision, moments=True)
        assert a.H == b.H
        assert np.array_equal(a.moments, b.moments)


def test_seeded_probes_passed_in_banded_f32():
    n, m, s, seed = 5000, 8, 32, 4
    vals = synth.band_diag_dominant(n, half_bw=16, seed=12, dtype=np.float32)
    u = 2.5 / n
    G = rng.probes(n, s, seed, "gaussian").astype(np.float32)
    b = vne.entropy_with_probes(dev(vals, torch.float32), dev(G, torch.float32), m, u=u,
                                precision="f32", moments=True, layout="dia")
    mu = O.chebyshev_moments(O.Dia(vals), G.astype(np.float64), u, m)
    sc = np.maximum(np.abs(mu).max(axis=1, keepdims=True), 1e-300)
    assert (np.abs(b.moments - mu) / sc).max() <= 2e-5
    assert rel(b.H, O.chebyshev_estimate_from_moments(mu, u)) < 2e-5


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("bf16x6", 1e-5)])
def test_eigenvector_probe_closed_forms(precision, tol):
    n, m = 256, 20
    R, p, psi = synth.dense_exp(n, 25.0, seed=7)
    u = 1.05 * p.max()
    g = psi[:, :1]  # eigenvector of p_1 (the largest eigenvalue)
    gt = torch.float64 if precision == "f64" else torch.float32
    c = vne.entropy_with_probes(dev(R), dev(g, gt), m, method="chebyshev", u=u,
                                precision=precision)
    assert rel(c.H, -float(O.cheb_fm(p[0], u, m))) < tol
    t = vne.entropy_with_probes(dev(R), dev(g, gt), m, method="taylor", u=u,
                                precision=precision)
    k = np.arange(1, m + 1)
    closed = np.log(1.0 / u) + float(np.sum(p[0] * (1.0 - p[0] / u) ** k / k))
    assert rel(t.H, closed) < tol


def test_unit_vector_and_zero_probes():
    n, m = 129, 12
    R, p, _ = synth.dense_exp(n, 20.0, seed=9)
    u = 1.02 * p.max()
    G = np.zeros((n, 4))
    G[0, 0] = 1.0
    G[64, 1] = 1.0
    G[n - 1, 2] = -1.0  # column 3 stays zero
    c = vne.entropy_with_probes(dev(R), dev(G), m, u=u, moments=True)
    mu = O.chebyshev_moments(R, G, u, m)
    np.testing.assert_allclose(c.moments, mu, rtol=1e-10, atol=1e-12)
    assert np.all(c.moments[:, 3] == 0.0)
    t = vne.entropy_with_probes(dev(R), dev(G), m, method="taylor", u=u, moments=True)
    tau = O.taylor_terms(R, G, u, m)
    np.testing.assert_allclose(t.moments, tau, rtol=1e-10, atol=1e-14)
    assert np.all(t.moments[:, 3] == 0.0)


def test_probe_block_type_and_shape_are_checked():
    R, _, _ = synth.dense_exp(64, 10.0, seed=1)
    with pytest.raises(ValueError):
        vne.entropy_with_probes(dev(R), dev(np.zeros((64, 2)), torch.float32), 4, u=0.5)
    with pytest.raises(ValueError):
        vne.entropy_with_probes(dev(R), dev(np.zeros((63, 2))), 4, u=0.5)
