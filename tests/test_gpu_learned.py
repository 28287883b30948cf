"""The learned moment correction on the GPU against the CPU FP64 oracle.

Tolerances (FP32 kernels against FP64 oracle arithmetic):
  spectral sampler   totals 1e-5 of s*n, H exact / H_16 1e-6 relative
  network forward    1e-5 of max |y|
  gradient           1e-4 of the largest entry of each parameter tensor
"""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.learned as L
import synth

pytestmark = pytest.mark.gpu

vne = pytest.importorskip("paper_1801_01072_gb300")
from paper_1801_01072_gb300 import learned  # noqa: E402


def spec_arrays(count, seed, n_lo=300, n_hi=1500):
    return synth.learned_sample_params(count, seed, n_lo, n_hi)


def oracle_sample(spec, b, m, s):
    p = synth.training_spectrum(int(spec["kind"][b]), int(spec["n"][b]), float(spec["a"][b]),
                                int(spec["ktop"][b]), float(spec["floor"][b]))
    u = float(spec["c"][b]) * p.max()
    tot = L.spectral_totals(p, u, m, s, int(spec["seed"][b]))
    H_low = L.chebyshev_from_totals(tot, u, s)
    return p, u, tot, H_low


@pytest.mark.parametrize("m", [15, 16, 64])
def test_spectral_sampler_matches_oracle(m):
    s = 16
    spec = spec_arrays(6, 11 + m)
    out = learned.spectral_samples(spec, m=m, s=s, totals=True)
    tot_g = out["totals"].cpu().numpy()
    for b in range(6):
        p, u, tot, H_low = oracle_sample(spec, b, m, s)
        n = p.size
        # FP32 polynomial recurrence: error grows with the degree k
        k = np.arange(m + 1)
        assert np.all(np.abs(tot_g[b] - tot) <= 2e-6 * (k + 1) * s * n)
        tol_H = 1e-6 * L.entropy(p)
        tol_low = (1e-5 if m <= 16 else 5e-5) * abs(H_low) + 1e-6  # grows with the degree
        assert abs(out["H_exact"][b].item() - L.entropy(p)) < tol_H
        assert abs(out["H_low"][b].item() - H_low) < tol_low
        f = L.features(tot, s, n, p.max(), u)
        np.testing.assert_allclose(out["features"][b].cpu().numpy(), f, rtol=1e-5, atol=1e-5)
        t = L.target(p, H_low, u)
        tol_t = 100.0 * (tol_H + tol_low) / (n * u) + 1e-6 * max(1.0, abs(t))
        assert abs(out["target"][b].item() - t) < tol_t


def test_network_forward_matches_oracle():
    theta = synth.mlp_init(3)
    X = np.random.default_rng(4).standard_normal((77, L.N_IN))
    y = learned.mlp_forward(torch.tensor(theta, dtype=torch.float32).cuda(),
                            torch.tensor(X, dtype=torch.float32).cuda()).cpu().numpy()
    ref, _ = L.forward(theta.astype(np.float32).astype(np.float64),
                       X.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("B", [1, 37, 64, 200])
def test_gradient_matches_oracle(B):
    rs = np.random.default_rng(B)
    theta = synth.mlp_init(7).astype(np.float32)
    X = rs.standard_normal((B, L.N_IN)).astype(np.float32)
    t = (0.1 * rs.standard_normal(B)).astype(np.float32)
    loss, g = learned.mlp_gradient(torch.tensor(theta).cuda(), torch.tensor(X).cuda(),
                                   torch.tensor(t).cuda())
    ref_loss, ref = L.backward(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    g = g.cpu().numpy()
    off = 0
    for i, o in L.LAYERS:
        for size in (o * i, o):
            seg, rseg = g[off:off + size], ref[off:off + size]
            assert np.abs(seg - rseg).max() <= 1e-4 * np.abs(rseg).max() + 1e-9, (off, size)
            off += size


def test_adam_step_matches_oracle():
    rs = np.random.default_rng(2)
    rows = 96
    theta = synth.mlp_init(9).astype(np.float32)
    X = rs.standard_normal((rows, L.N_IN)).astype(np.float32)
    t = (0.1 * rs.standard_normal(rows)).astype(np.float32)
    th = torch.tensor(theta).cuda()
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    h = vne._handle(0)
    import ctypes as C
    loss = C.c_double()
    Xd, td = torch.tensor(X).cuda(), torch.tensor(t).cuda()  # kept alive across the call
    torch.cuda.synchronize()
    # batch = rows: the whole (permuted) data set, so the gradient is the oracle's
    st = h.lib.vne_mlp_train_step(h.h, C.c_void_p(th.data_ptr()), C.c_void_p(m.data_ptr()),
                                  C.c_void_p(v.data_ptr()), 1, 1e-3, C.c_void_p(Xd.data_ptr()),
                                  C.c_void_p(td.data_ptr()), rows, rows, 0, 5, C.byref(loss), None)
    assert st == 0
    ref_loss, g = L.backward(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    new, _, _ = L.adam_step(theta.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    assert abs(loss.value - ref_loss) <= 1e-5 * ref_loss
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    np.testing.assert_allclose(th.cpu().numpy()[big], new[big], rtol=0, atol=2e-6)


def test_training_reduces_error_on_held_out_spectra():
    s = 128
    train_spec = synth.learned_sample_params(20000, 1)
    data = learned.spectral_samples(train_spec, s=s)
    theta0 = torch.tensor(synth.mlp_init(1), dtype=torch.float32).cuda()
    theta, hist = learned.train(theta0, data["features"], data["target"], epochs=8, batch=512,
                                lr=2e-3, report_every=50)
    X, t = data["features"][:4096], data["target"][:4096]
    loss0, _ = learned.mlp_gradient(theta0, X, t)
    loss1, _ = learned.mlp_gradient(theta, X, t)
    # The targets carry the probe noise of H_16, which no function of the
    # spectrum predicts.  Its variance is half the mean squared difference of
    # two targets of the same spectra drawn with other probe seeds; the
    # network must remove at least half of the loss above that floor.
    sub = {k: np.asarray(v)[:4096] for k, v in train_spec.items()}
    sub2 = dict(sub, seed=(sub["seed"] ^ np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64))
    t2 = learned.spectral_samples(sub2, s=s)["target"]
    floor = 0.5 * float(((t - t2).double() ** 2).mean())
    assert loss1 < loss0
    assert loss0 - loss1 >= 0.5 * (loss0 - floor), (loss0, loss1, floor)
    for n_lo, n_hi in ((1024, 4096), (8192, 8192)):
        test = learned.spectral_samples(synth.learned_sample_params(1000, 99, n_lo, n_hi), s=s)
        corr = learned.mlp_forward(theta, test["features"]).double()
        sp = synth.learned_sample_params(1000, 99, n_lo, n_hi)
        n = torch.tensor(sp["n"], dtype=torch.float64).cuda()
        # u = c p_1, with ln(u)/10 the last feature
        u = torch.exp(10.0 * test["features"][:, 18].double())
        H = test["H_exact"]
        plain = ((test["H_low"] - H).abs() / H).mean().item()
        fixed = ((test["H_low"] + corr * n * u / 100.0 - H).abs() / H).mean().item()
        assert fixed < 0.5 * plain, (n_lo, plain, fixed)


def test_sampler_distribution_matches_real_estimator():
    # the totals of the real GPU estimator (FP64, Gaussian probes) on
    # R = Psi diag(p) Psi^T scatter around s * sum_i T_k(x_i), like the sampler's
    n, s, m = 384, 32, 16
    p = synth.training_spectrum(1, n, 1.3, 100, 1e-8)
    R = synth.dense_density(synth.haar_orthogonal(n, 5), p)
    u = 1.05 * p.max()
    expect = s * np.polynomial.chebyshev.chebvander(2 * p / u - 1, m).sum(axis=0)
    reps = 24
    real = np.array([vne.entropy_chebyshev(torch.tensor(R).cuda(), m, s, seed=100 + r,
                                           probe="gaussian", u=u, moments=True).moments.sum(axis=1)
                     for r in range(reps)])
    spec = {k: np.repeat(np.asarray(v)[:1], reps) for k, v in dict(
        kind=np.int32([1]), n=np.int32([n]), a=np.float32([1.3]), ktop=np.int32([100]),
        floor=np.float32([1e-8]), c=np.float32([1.05])).items()}
    spec["seed"] = np.arange(1, reps + 1, dtype=np.uint64)
    samp = learned.spectral_samples(spec, m=m, s=s, totals=True)["totals"].cpu().numpy()
    for arr in (real, samp):
        se = arr.std(axis=0, ddof=1) / np.sqrt(reps)
        assert np.all(np.abs(arr.mean(axis=0) - expect) <= 5 * se + 1e-6 * s * n)


def test_learned_estimator_on_matrices():
    # the corrected estimate of real matrices: H_plain equals the plain
    # degree-16 estimator; the correction brings it closer to the exact H
    s = 128
    spec = synth.learned_sample_params(12000, 3)
    data = learned.spectral_samples(spec, s=s)
    theta, _ = learned.train(torch.tensor(synth.mlp_init(2), dtype=torch.float32).cuda(),
                             data["features"], data["target"], epochs=6, batch=512, lr=2e-3)
    errs_plain, errs_fixed = [], []
    for i, (kind, a, ktop) in enumerate([(0, 300.0, 0), (1, 1.5, 500), (1, 1.2, 800), (0, 80.0, 0)]):
        n = 2048
        p = synth.training_spectrum(kind, n, a, ktop, 1e-8)
        R = torch.tensor(synth.dense_density(synth.haar_orthogonal(n, 10 + i), p)).cuda()
        res = learned.entropy_chebyshev_learned(R, theta, s=s, seed=7 + i, precision="f64")
        plain = vne.entropy_chebyshev(R, 16, s, seed=7 + i, probe="gaussian", u_scale=1.05)
        assert res.H_plain == plain.H
        H = L.entropy(p)
        errs_plain.append(abs(res.H_plain - H) / H)
        errs_fixed.append(abs(res.H - H) / H)
    assert np.mean(errs_fixed) < np.mean(errs_plain)
