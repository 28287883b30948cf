"""One estimate split by probe range (vne_params.probe_offset) and recombined
on the device (vne_combine_moments), against the single call.

Every probe's moments depend only on R, u and that probe (Lemma thm:trace
makes the estimate their mean), so two calls on probes [0, s1) and [s1, s)
must give the single call's per-probe moments, and the combination of the
gathered moments its estimate.  On the FP64 path with one K slice per
product (n >= 9760 rows: 305 row tiles fill the GPU without a K split) each
moment is the same chain of FMAs in both cases, so the equality is exact.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import rng

pytestmark = pytest.mark.gpu

vne = pytest.importorskip("paper_1801_01072_gb300")


def psd_matrix(n, k, seed):
    """(A A^T + I) / trace with A n x k Gaussian: a symmetric positive
    definite unit-trace R, built on the GPU."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    A = torch.randn(n, k, generator=g, device="cuda", dtype=torch.float64)
    R = A @ A.T + torch.eye(n, device="cuda", dtype=torch.float64)
    return (R / torch.trace(R)).contiguous()


def split_calls(R, m, s, s1, **kw):
    a = vne.entropy_both(R, m, s1, moments=True, probe_offset=0, **kw)
    b = vne.entropy_both(R, m, s - s1, moments=True, probe_offset=s1, **kw)
    assert a.u == b.u
    mc = np.concatenate([a.moments_chebyshev, b.moments_chebyshev], axis=1)
    mt = np.concatenate([a.moments_taylor, b.moments_taylor], axis=1)
    return mc, mt, a.u


def test_probe_split_fp64_is_exact():
    n, m, s, s1 = 9760, 6, 64, 21
    R = psd_matrix(n, 64, 3)
    kw = dict(seed=11, probe="gaussian", precision="f64", power_iters=30)
    one = vne.entropy_both(R, m, s, moments=True, **kw)
    mc, mt, u = split_calls(R, m, s, s1, **kw)
    assert u == one.u
    assert np.array_equal(mc, one.moments_chebyshev)
    assert np.array_equal(mt, one.moments_taylor)
    Hc, Ht = vne.combine_moments(m, s, u, mc, mt)
    assert Hc == one.H_chebyshev and Ht == one.H_taylor


def test_probe_split_bf16_matches_single_call():
    n, m, s, s1 = 4096, 12, 128, 64
    R = psd_matrix(n, 256, 4)
    kw = dict(seed=5, probe="gaussian", precision="bf16", power_iters=30)
    one = vne.entropy_both(R, m, s, moments=True, **kw)
    mc, mt, u = split_calls(R, m, s, s1, **kw)
    for got, ref in ((mc, one.moments_chebyshev), (mt, one.moments_taylor)):
        sc = np.abs(ref).max(axis=1, keepdims=True)
        assert (np.abs(got - ref) / sc).max() <= 1e-9
    Hc, Ht = vne.combine_moments(m, s, u, mc, mt)
    assert abs(Hc - one.H_chebyshev) <= 1e-9 * abs(one.H_chebyshev)
    assert abs(Ht - one.H_taylor) <= 1e-9 * abs(one.H_taylor)


def test_probe_offset_draws_the_later_probes():
    # the moments of probes j0.. of a call equal the oracle's on columns j0..
    n, m, s, j0 = 300, 5, 7, 9
    R = psd_matrix(n, 20, 5).cpu().numpy()
    u = 1.1 * float(np.linalg.eigvalsh(R).max())
    res = vne.entropy_chebyshev(torch.as_tensor(R).cuda(), m, s, seed=2, probe="rademacher",
                                precision="f64", u=u, moments=True, probe_offset=j0)
    G = rng.probes(n, j0 + s, 2, "rademacher")[:, j0:]
    mu = O.chebyshev_moments(R, G, u, m)
    assert np.abs(res.moments - mu).max() <= 1e-10 * np.abs(mu).max()


def test_combine_moments_checks_its_arguments():
    with pytest.raises(vne.VneError) as e:
        vne.combine_moments(3, 2, 1.5, np.zeros((4, 2)))
    assert e.value.status == 3
    with pytest.raises(ValueError):
        vne.combine_moments(3, 2, 0.5, np.zeros((3, 2)))
