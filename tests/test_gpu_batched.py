"""Batched estimates of uneven matrices (one call, concurrent streams, CUDA
graph replay) against the single calls and the oracle.

These tests pin the stream path (VNE_BATCH_PERSISTENT=0), whose per-matrix
kernels are those of the single calls, so results agree bit for bit; the
persistent recurrence of BF16 batches is tested in
test_gpu_batched_persistent.py."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

vne = pytest.importorskip("paper_1801_01072_gb300")


@pytest.fixture(autouse=True)
def stream_path(monkeypatch):
    monkeypatch.setenv("VNE_BATCH_PERSISTENT", "0")


def mats(sizes, seed0=0):
    out = []
    for i, n in enumerate(sizes):
        R, p, _ = synth.dense_exp(n, max(4.0, n / 10), seed=seed0 + i)
        out.append((torch.tensor(R).cuda(), R, p))
    return out


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("precision,method", [("f64", "both"), ("bf16", "chebyshev"),
                                              ("f32", "taylor")])
def test_batched_equals_single_calls(use_graph, precision, method):
    sizes = [64, 200, 333, 97, 512, 130, 256, 40, 300, 150]
    ms = mats(sizes)
    m, s, seed = 12, 16, 9
    hc, ht, u = vne.entropy_batched([t for t, _, _ in ms], m, s, seed=seed, probe="gaussian",
                                    precision=precision, method=method, use_graph=use_graph)
    kw = dict(seed=seed, probe="gaussian", precision=precision)
    for i, (t, R, p) in enumerate(ms):
        # the same estimator set as the batch (the fused column count decides
        # the tiling, hence the rounding order)
        if method == "both":
            one = vne.entropy_both(t, m, s, **kw)
            assert (hc[i], ht[i], u[i]) == (one.H_chebyshev, one.H_taylor, one.u), i
        elif method == "chebyshev":
            one = vne.entropy_chebyshev(t, m, s, **kw)
            assert (hc[i], u[i]) == (one.H, one.u), (i, hc[i], one.H)
        else:
            one = vne.entropy_taylor(t, m, s, **kw)
            assert (ht[i], u[i]) == (one.H, one.u), (i, ht[i], one.H)
    if precision == "f64":
        for i, (t, R, p) in enumerate(ms[:3]):
            ref = O.estimate(R, "chebyshev", m, s, seed, "gaussian", power_iters=30)
            assert abs(hc[i] - ref["H"]) <= 1e-10 * abs(ref["H"])


def test_graph_replay_and_recapture():
    ms = mats([128, 256, 77], seed0=20)
    ts = [t for t, _, _ in ms]
    a = vne.entropy_batched(ts, 10, 8, seed=3, precision="bf16")[0]
    b = vne.entropy_batched(ts, 10, 8, seed=3, precision="bf16")[0]   # replay
    assert np.array_equal(a, b)
    c = vne.entropy_batched(ts, 10, 8, seed=4, precision="bf16")[0]   # new key: recapture
    d = vne.entropy_batched(ts, 10, 8, seed=4, precision="bf16", use_graph=False)[0]
    assert np.array_equal(c, d) and not np.array_equal(a, c)
    # different matrices with the same shapes: recaptured, not stale
    ms2 = mats([128, 256, 77], seed0=40)
    e = vne.entropy_batched([t for t, _, _ in ms2], 10, 8, seed=3, precision="bf16")[0]
    f = [vne.entropy_chebyshev(t, 10, 8, seed=3, precision="bf16").H for t, _, _ in ms2]
    assert np.array_equal(e, np.array(f))


def test_batched_mixed_layouts_and_errors():
    n = 3000
    vals = synth.band_diag_dominant(n, 16, 0.02, seed=2, dtype=np.float64)
    band = torch.tensor(vals).cuda()
    dense, _, _ = mats([180])[0]
    hc, _, _ = vne.entropy_batched([dense, band], 8, 6, seed=1, precision="f64",
                                   layouts=["dense", "dia"])
    one = vne.entropy_chebyshev(band, 8, 6, seed=1, precision="f64", layout="dia")
    assert hc[1] == one.H
    with pytest.raises(vne.VneError):
        vne.entropy_batched([dense, band], 8, 6, seed=1, precision="bf16",
                            layouts=["dense", "dia"])   # banded BF16 is not supported


def test_autotune_picks_a_candidate_and_results_hold():
    t, R, p = mats([1024], seed0=60)[0]
    shape, us = vne.autotune(t, 10, 32, precision="bf16", method="chebyshev", seed=2)
    BN, CM, CN, ks = shape
    assert BN % 32 == 0 and 32 <= BN <= 256 and CM == CN == 1 and ks in (1, 2) and us > 0
    res = vne.entropy_chebyshev(t, 10, 32, seed=2, probe="gaussian", precision="bf16")
    from oracle import rng
    G = rng.probes(1024, 32, 2, "gaussian")
    ref = O.chebyshev_estimate_from_moments(O.chebyshev_moments(R, G, res.u, 10), res.u)
    assert abs(res.H - ref) <= 1e-3 * abs(ref)


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
def test_batched_large_matrices_equal_single_calls(precision):
    """n >= 2048: the single calls run the power method's products in one
    cooperative launch, the batched call phase by phase on a smaller grid;
    the bits agree (every sum has a fixed order whatever the grid)."""
    sizes = [2048, 2300, 3001, 700, 4096]
    ms = mats(sizes, seed0=80)
    m, s, seed = 10, 8, 5
    hc, _, u = vne.entropy_batched([t for t, _, _ in ms], m, s, seed=seed, probe="gaussian",
                                   precision=precision)
    for i, (t, R, p) in enumerate(ms):
        one = vne.entropy_chebyshev(t, m, s, seed=seed, probe="gaussian", precision=precision)
        assert (hc[i], u[i]) == (one.H, one.u), (i, sizes[i], hc[i], one.H, u[i], one.u)
