"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Every comparison runs both sides on the same seeded matrix, the same probes
(each side draws them from its own SplitMix64 code) and the same u.
Tolerances (relative, on the estimate H and on each moment):
  FP64 path            1e-10  (both sides FP64; only the summation order differs)
  FP32 banded path     2e-5   (FP32 products over <= 33 diagonals, FP64 moments)
  bf16x6 dense path    1e-6   (three bf16 pieces of R and Y, six products; the
                              moments 1e-5, bounded by the FP32 master of Y)
  bf16x3 dense path    1e-5   (about 16 significant bits per product; moments 5e-4)
  BF16 dense path      1e-3   (8-bit significands; the bar for the mixed path)
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


def moments_close(got, ref, rtol, scale=None):
    """Compare per-probe moments relative to the magnitude of each row."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    sc = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-300) if scale is None else scale
    err = np.abs(got - ref) / sc
    assert err.max() <= rtol, f"max scaled moment error {err.max():.3e} > {rtol}"


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


# ---------------------------------------------------------------------------
# probe generator
# ---------------------------------------------------------------------------

def test_rademacher_stream_bit_exact_1e6_draws():
    n, s, seed = 100_003, 10, 0xC0FFEE
    got = vne.probe_block(n, s, seed, "rademacher").cpu().numpy()
    assert np.array_equal(got, rng.rademacher(n, s, seed))


def test_gaussian_stream_matches():
    n, s, seed = 4099, 7, 12345
    got = vne.probe_block(n, s, seed, "gaussian").cpu().numpy()
    ref = rng.gaussian(n, s, seed)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------
# dense FP64 (SIMT) path: tiles 32 x 32, split-K, ragged edges
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 17, 64, 127, 128, 129, 513])
@pytest.mark.parametrize("s", [1, 3, 50])
def test_dense_f64_chebyshev_and_taylor(n, s):
    R, p, _ = synth.dense_exp(n, max(n / 5.0, 1.0), seed=100 + n)
    u = min(1.0, 1.05 * p.max())
    for m in (1, 2, 3, 20):
        G = rng.probes(n, s, 7, "gaussian")
        rc = vne.entropy_chebyshev(dev(R), m, s, seed=7, probe="gaussian", u=u, moments=True)
        mu = O.chebyshev_moments(R, G, u, m)
        moments_close(rc.moments, mu, 1e-10)
        assert rel(rc.H, O.chebyshev_estimate_from_moments(mu, u)) < 1e-10
        assert rel(rc.H, O.chebyshev_estimate_clenshaw(R, G, u, m)) < 1e-10
        rt = vne.entropy_taylor(dev(R), m, s, seed=7, probe="gaussian", u=u, moments=True)
        tau = O.taylor_terms(R, G, u, m)
        moments_close(rt.moments, tau, 1e-10)
        assert rel(rt.H, O.taylor_estimate_from_terms(tau, u)) < 1e-10


def test_dense_f64_both_equals_separate_calls():
    R, p, _ = synth.dense_exp(200, 40.0, seed=3)
    b = vne.entropy_both(dev(R), 9, 11, seed=5, moments=True)
    c = vne.entropy_chebyshev(dev(R), 9, 11, seed=5, moments=True)
    t = vne.entropy_taylor(dev(R), 9, 11, seed=5, moments=True)
    assert rel(b.H_chebyshev, c.H) < 1e-12 and rel(b.H_taylor, t.H) < 1e-12
    assert b.u == c.u == t.u


@pytest.mark.parametrize("q", [1, 3])
def test_power_method_f64(q):
    R, p, _ = synth.dense_exp(300, 30.0, seed=9)
    lam = vne.lambda_max(dev(R), power_iters=12, power_trials=q, seed=4)
    ref, _ = O.power_method(R, rng.power_start(300, q, 4), 12)
    assert rel(lam, ref) < 1e-12
    assert p.max() / 6 <= lam <= p.max() * (1 + 1e-12)  # Lemma lem:power bracket


@pytest.mark.parametrize("n,q", [(300, 1), (1024, 1), (2500, 1), (1024, 3)])
def test_power_method_tensor_core_path(n, q):
    """The BF16 path's power method (products with the bf16 copy of R, FP32
    accumulation, FP64 Rayleigh quotient) stays within the BF16 path's 1e-3
    of the FP64 power method.  (After t = 30 products the iterate is not
    converged, so the Rayleigh quotient moves to first order with the
    rounding of R; the deviation, ~1e-4, is far below the method's own gap to
    p_1.)"""
    R, p, _ = synth.dense_exp(n, n / 10.0, seed=40 + n)
    lam = vne.lambda_max(dev(R), power_iters=30, power_trials=q, seed=2, precision="bf16")
    ref, _ = O.power_method(R, rng.power_start(n, q, 2), 30)
    assert rel(lam, ref) < 1e-3
    assert abs(lam - ref) < 0.1 * (p.max() - ref)  # well inside the power method's own error


def test_dense_n512_exp_spectrum_full_pipeline():
    """n = 512, p_i ~ exp(-i/50), m = 20, s = 50 Rademacher, t = 30, FP64."""
    R, p, _ = synth.dense_exp(512, 50.0, seed=1)
    res = vne.entropy_chebyshev(dev(R), 20, 50, seed=11, probe="rademacher", power_iters=30,
                                moments=True)
    ref = O.estimate(R, "chebyshev", 20, 50, 11, "rademacher", power_iters=30)
    assert rel(res.u, ref["u"]) < 1e-12
    assert rel(res.H, ref["H"]) < 1e-10
    # against the exact entropy: the truncation bound (eq. PD2) plus 5 sigma of
    # the Rademacher quadratic form
    H = O.entropy_of_spectrum(p)
    nte = O.nte_chebyshev(p, res.u, 20)
    a = -O.cheb_fm(p, res.u, 20)
    A = (synth.haar_orthogonal(512, 1) * a) @ synth.haar_orthogonal(512, 1).T
    sigma = np.sqrt(2 * ((A ** 2).sum() - (np.diag(A) ** 2).sum()) / 50)
    assert abs(res.H - nte) < 5 * sigma
    assert abs(nte - H) <= 512 * res.u / (2 * 20 * 21)
    rt = vne.entropy_taylor(dev(R), 20, 50, seed=11, probe="rademacher", power_iters=30)
    reft = O.estimate(R, "taylor", 20, 50, 11, "rademacher", power_iters=30)
    assert rel(rt.H, reft["H"]) < 1e-10


# ---------------------------------------------------------------------------
# dense FP32 (SIMT) path
# ---------------------------------------------------------------------------

def test_dense_f32_parity():
    R, p, _ = synth.dense_exp(300, 30.0, seed=4)
    u = p.max()
    G = rng.probes(300, 13, 2, "rademacher")
    res = vne.entropy_chebyshev(dev(R), 12, 13, seed=2, u=u, precision="f32", moments=True)
    ref = O.chebyshev_estimate_from_moments(O.chebyshev_moments(R, G, u, 12), u)
    assert rel(res.H, ref) < 1e-5


# ---------------------------------------------------------------------------
# banded (DIA) path: FP32 and FP64, every compiled window, chunk edges
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,hb", [(1, 1), (2, 1), (17, 2), (300, 4), (1000, 8), (5000, 16),
                                  (100_003, 16), (273, 16), (545, 16)])
@pytest.mark.parametrize("s", [1, 2, 3, 64])
def test_dia_f32_parity(n, hb, s):
    vals = synth.band_diag_dominant(n, half_bw=min(hb, max(n - 1, 0)) or 1, seed=n,
                                    dtype=np.float32)
    Rop = O.Dia(vals)
    ev_hi = 2.5 / n
    u = min(1.0, ev_hi)
    m = 6
    G = rng.probes(n, s, 3, "rademacher")
    rc = vne.entropy_chebyshev(dev(vals), m, s, seed=3, u=u, precision="f32", layout="dia",
                               moments=True)
    mu = O.chebyshev_moments(Rop, G, u, m)
    moments_close(rc.moments, mu, 2e-5)
    assert rel(rc.H, O.chebyshev_estimate_from_moments(mu, u)) < 2e-5
    rt = vne.entropy_taylor(dev(vals), m, s, seed=3, u=u, precision="f32", layout="dia",
                            moments=True)
    tau = O.taylor_terms(Rop, G, u, m)
    moments_close(rt.moments, tau, 2e-5)


def test_dia_gaussian_probes_and_f64():
    n = 3001
    vals = synth.band_diag_dominant(n, half_bw=16, seed=5, dtype=np.float64)
    u = 2.5 / n
    G = rng.probes(n, 5, 8, "gaussian")
    for prec, tol in (("f64", 1e-10), ("f32", 2e-5)):
        v = vals if prec == "f64" else vals.astype(np.float32)
        rc = vne.entropy_chebyshev(dev(v), 7, 5, seed=8, probe="gaussian", u=u, precision=prec,
                                   layout="dia", moments=True)
        mu = O.chebyshev_moments(O.Dia(v), G, u, 7)
        moments_close(rc.moments, mu, tol)


def test_dia_power_method():
    n = 20_000
    vals = synth.band_diag_dominant(n, half_bw=16, seed=6, dtype=np.float32)
    lam = vne.lambda_max(dev(vals), power_iters=30, seed=1, precision="f32", layout="dia")
    ref, _ = O.power_method(O.Dia(vals), rng.power_start(n, 1, 1), 30)
    assert rel(lam, ref) < 1e-5


def test_poisson_tridiagonal_closed_form():
    """Section 6: tridiag(-1,2,-1)/(2n), u = lambda_max from eq. trig_eigs."""
    n = 5000
    vals = synth.band_poisson(n)
    lam = synth.spectrum_poisson(n)
    u = lam.max()
    res = vne.entropy_chebyshev(dev(vals), 5, 50, seed=2, probe="gaussian", u=u,
                                layout="dia")
    G = rng.probes(n, 50, 2, "gaussian")
    ref = O.chebyshev_estimate_from_moments(O.chebyshev_moments(O.Dia(vals), G, u, 5), u)
    assert rel(res.H, ref) < 1e-10
    H = O.entropy_of_spectrum(lam)
    assert rel(res.H, H) < 0.05


def test_band_1e7_sampled_probe():
    """n = 10^7, half-bandwidth 16, s = 64 Rademacher, FP32: the launch
    configuration of the banded workload; probe 0's moments against the
    oracle (the moments of each probe are independent)."""
    n, s, m = 10_000_000, 64, 4
    vals = synth.band_diag_dominant(n, half_bw=16, seed=3, dtype=np.float32)
    dv = dev(vals)
    u = 1.6 / n
    rc = vne.entropy_chebyshev(dv, m, s, seed=9, u=u, precision="f32", layout="dia",
                               moments=True)
    g0 = rng.probes(n, 1, 9, "rademacher")  # probe 0 is the first column block
    mu = O.chebyshev_moments(O.Dia(vals), g0, u, m)
    np.testing.assert_allclose(rc.moments[:, :1], mu, rtol=2e-5)


# ---------------------------------------------------------------------------
# dense tensor-core path (tcgen05): BF16 and bf16x3
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [64, 128, 129, 300, 513])
@pytest.mark.parametrize("s", [1, 50, 128])
def test_dense_tc_parity(n, s):
    R, p, _ = synth.dense_exp(n, max(n / 8.0, 2.0), seed=200 + n)
    u = min(1.0, 1.02 * p.max())
    m = 10
    G = rng.probes(n, s, 4, "gaussian")
    mu = O.chebyshev_moments(R, G, u, m)
    Href = O.chebyshev_estimate_from_moments(mu, u)
    tau = O.taylor_terms(R, G, u, m)
    Htref = O.taylor_estimate_from_terms(tau, u)
    for prec, tol, mtol in (("bf16", 1e-3, None), ("bf16x3", 1e-5, 5e-4), ("bf16x6", 1e-6, 1e-5)):
        b = vne.entropy_both(dev(R), m, s, seed=4, probe="gaussian", u=u, precision=prec,
                             moments=True)
        assert rel(b.H_chebyshev, Href) < tol, (prec, b.H_chebyshev, Href)
        assert rel(b.H_taylor, Htref) < tol, (prec, b.H_taylor, Htref)
        if mtol is not None:
            moments_close(b.moments_chebyshev, mu, mtol)
            moments_close(b.moments_taylor, tau, mtol)
        c = vne.entropy_chebyshev(dev(R), m, s, seed=4, probe="gaussian", u=u, precision=prec)
        assert rel(c.H, Href) < tol


# ---------------------------------------------------------------------------
# errors, host memory, edge cases
# ---------------------------------------------------------------------------

def test_host_memory_matrix_equals_device():
    R, p, _ = synth.dense_exp(256, 30.0, seed=8)
    a = vne.entropy_chebyshev(dev(R), 8, 16, seed=1)
    b = vne.entropy_chebyshev(torch.as_tensor(R).pin_memory(), 8, 16, seed=1)
    assert a.H == b.H and a.u == b.u


def test_error_statuses():
    R, p, _ = synth.dense_exp(64, 10.0, seed=8)
    with pytest.raises(vne.VneError) as e:
        vne.entropy_chebyshev(dev(R), 0, 4)
    assert e.value.status == 1
    with pytest.raises(vne.VneError) as e:
        vne.entropy_chebyshev(dev(R), 4, 4, u=1.5)
    assert e.value.status == 3
    with pytest.raises(vne.VneError) as e:
        vne.entropy_chebyshev(dev(2.0 * R), 4, 4, check_trace=True)
    assert e.value.status == 2
    ok = vne.entropy_chebyshev(dev(R), 4, 4, check_trace=True)
    assert np.isfinite(ok.H)
    with pytest.raises(vne.VneError) as e:
        vne.entropy_chebyshev(dev(R), 4, 4, precision="bf16", layout="dia")
    assert e.value.status in (1, 8)


def test_maximally_mixed_on_gpu():
    n = 96
    R = np.eye(n) / n
    t = vne.entropy_taylor(dev(R), 10, 8, seed=3, probe="gaussian")
    assert abs(t.H - np.log(n)) < 1e-12
    assert abs(t.u - 1.0 / n) < 1e-15


def test_launches_are_counted():
    h = vne._handle(0)
    before = h.launch_count()
    R, p, _ = synth.dense_exp(64, 10.0, seed=8)
    vne.entropy_chebyshev(dev(R), 4, 4)
    assert h.launch_count() > before


def test_bounded_wait_times_out_and_context_survives():
    # a wait that nothing satisfies ends with VNE_ERR_TIMEOUT after the
    # deadline; the next call on the same handle and stream works
    import time
    h = vne._handle(0)
    t0 = time.perf_counter()
    st = h.lib.vne_selftest_timeout(h.h, None)
    dt = time.perf_counter() - t0
    assert st == 6, st  # VNE_ERR_TIMEOUT
    assert 1.5 < dt < 30.0
    R, p, _ = synth.dense_exp(64, 10.0, seed=1)
    res = vne.entropy_chebyshev(dev(R), 6, 4, seed=1, precision="f64")
    assert np.isfinite(res.H)


def _bf16_round(a):
    """Round to bf16 (through FP32, round-to-nearest-even), as the library's
    conversion of R does; returns FP64."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _split2(a, fp64_residual):
    """The first two bf16 pieces of the split modes' copy of R: bf16x3 splits
    R rounded to FP32 (FP32 residual), bf16x6 takes the residual in FP64."""
    if fp64_residual:
        h = _bf16_round(a)
        return h + _bf16_round(np.asarray(a, dtype=np.float64) - h)
    v = np.asarray(a, dtype=np.float32).astype(np.float64)
    h = _bf16_round(v)
    return h + _bf16_round(v - h)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_power_method_split_modes_against_oracle(prec):
    """The split modes' power method (the persistent kernel on the first two
    bf16 pieces, R_0 + R_1 exact in FP32) against Algorithm alg:power in
    FP64 on the same two-piece R, and against FP64 on R itself."""
    n = 3000
    R, p, _ = synth.dense_exp(n, n / 12.0, seed=77)
    lam = vne.lambda_max(dev(R), power_iters=30, seed=3, precision=prec)
    ref, _ = O.power_method(_split2(R, prec == "bf16x6"), rng.power_start(n, 1, 3), 30)
    assert rel(lam, ref) < 2e-6, (lam, ref)
    exact, _ = O.power_method(R, rng.power_start(n, 1, 3), 30)
    assert rel(lam, exact) < 1e-6, (lam, exact)


@pytest.mark.parametrize("n", [2048, 2049, 4100])
def test_power_method_bf16_persistent_against_oracle(n):
    """The BF16 path's power method (all products in one launch over the upper
    triangle of the bf16 copy of R) against Algorithm alg:power in FP64 on the
    same bf16-rounded R: only the FP32 summation order differs."""
    R, p, _ = synth.dense_exp(n, n / 12.0, seed=70 + n)
    lam = vne.lambda_max(dev(R), power_iters=30, seed=3, precision="bf16")
    ref, _ = O.power_method(_bf16_round(R), rng.power_start(n, 1, 3), 30)
    assert rel(lam, ref) < 2e-6, (lam, ref)
