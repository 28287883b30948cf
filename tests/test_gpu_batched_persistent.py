"""The persistent recurrence of BF16 batches (one launch for every step of
every matrix, work items in dependency order) through vne_entropy_batched.

Each estimate is checked against the oracle's same-probe estimate at the u
the batch returns (BF16 tolerance 1e-3, matrices of order >= 64), against the
stream path on the same batch (the same products in another FP32 summation
order: 1e-4 on H, 1e-5 on u), and for replay determinism (bit-identical).  The
power method of the batch (its own persistent launch) is checked against the
oracle's FP64 power method at the BF16 path's 1e-3.  Sizes cover one
tile (n <= 128), ragged last tiles and the largest batch matrices (4096);
L2 budgets small enough to force many rounds and large enough for one."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle import rng

pytestmark = pytest.mark.gpu

vne = pytest.importorskip("paper_1801_01072_gb300")


def mats(sizes, seed0=0):
    out = []
    for i, n in enumerate(sizes):
        R, p, _ = synth.dense_exp(n, max(4.0, n / 10), seed=seed0 + i)
        out.append((torch.tensor(R).cuda(), R, p))
    return out


def oracle_H(R, method, m, s, seed, u):
    G = rng.probes(R.shape[0], s, seed, "gaussian")
    hc = ht = None
    if method in ("chebyshev", "both"):
        hc = O.chebyshev_estimate_from_moments(O.chebyshev_moments(R, G, u, m), u)
    if method in ("taylor", "both"):
        ht = O.taylor_estimate_from_terms(O.taylor_terms(R, G, u, m), u)
    return hc, ht


@pytest.mark.parametrize("method,s", [("chebyshev", 32), ("both", 32), ("taylor", 16),
                                      ("chebyshev", 50)])
@pytest.mark.parametrize("l2_mb", ["0.25", "64"])
def test_persistent_batch_vs_oracle_and_stream_path(monkeypatch, method, s, l2_mb):
    sizes = [64, 200, 333, 97, 512, 130, 256, 1000, 300, 150, 128, 129]
    ms = mats(sizes, seed0=100)
    m, seed = 12, 9
    ts = [t for t, _, _ in ms]
    monkeypatch.setenv("VNE_BATCH_L2_MB", l2_mb)
    monkeypatch.setenv("VNE_BATCH_MIN_TILES", "0")
    hc, ht, u = vne.entropy_batched(ts, m, s, seed=seed, probe="gaussian", precision="bf16",
                                    method=method)
    monkeypatch.setenv("VNE_BATCH_PERSISTENT", "0")
    hc0, ht0, u0 = vne.entropy_batched(ts, m, s, seed=seed, probe="gaussian", precision="bf16",
                                       method=method)
    # the power method runs in the batch's own persistent launch: the same
    # bf16 products in another FP32 summation order
    np.testing.assert_allclose(u, u0, rtol=1e-5)
    for i, (t, R, p) in enumerate(ms):
        rc, rt = oracle_H(R, method, m, s, seed, u[i])
        if rc is not None:
            assert abs(hc[i] - rc) <= 1e-3 * abs(rc), (i, sizes[i], hc[i], rc)
            assert abs(hc[i] - hc0[i]) <= 1e-4 * abs(hc0[i]), (i, hc[i], hc0[i])
        if rt is not None:
            assert abs(ht[i] - rt) <= 1e-3 * abs(rt), (i, sizes[i], ht[i], rt)
            assert abs(ht[i] - ht0[i]) <= 1e-4 * abs(ht0[i]), (i, ht[i], ht0[i])


def test_persistent_batch_large_matrices_and_replay():
    sizes = [4096, 2048, 700, 3001, 256]
    ms = mats(sizes, seed0=140)
    m, s, seed = 10, 32, 5
    ts = [t for t, _, _ in ms]
    a = vne.entropy_batched(ts, m, s, seed=seed, probe="gaussian", precision="bf16")
    b = vne.entropy_batched(ts, m, s, seed=seed, probe="gaussian", precision="bf16")  # replay
    c = vne.entropy_batched(ts, m, s, seed=seed, probe="gaussian", precision="bf16",
                            use_graph=False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[0], c[0])
    for i, (t, R, p) in enumerate(ms):
        rc, _ = oracle_H(R, "chebyshev", m, s, seed, a[2][i])
        assert abs(a[0][i] - rc) <= 1e-3 * abs(rc), (i, sizes[i], a[0][i], rc)


def test_persistent_batch_many_small_matrices():
    """256 matrices of n in [64, 400]: rounds with hundreds of matrices."""
    r = np.random.default_rng(3)
    sizes = [int(x) for x in np.floor(64 * (400 / 64) ** r.random(256))]
    ms = mats(sizes, seed0=300)
    m, s, seed = 8, 32, 2
    hc, _, u = vne.entropy_batched([t for t, _, _ in ms], m, s, seed=seed, probe="gaussian",
                                   precision="bf16")
    for i in range(0, 256, 17):
        rc, _ = oracle_H(ms[i][1], "chebyshev", m, s, seed, u[i])
        assert abs(hc[i] - rc) <= 1e-3 * abs(rc), (i, sizes[i], hc[i], rc)


def test_persistent_power_method_vs_oracle():
    from oracle import rng as R_
    sizes = [64, 129, 1000, 2048, 4096, 300]
    ms = mats(sizes, seed0=500)
    _, _, u = vne.entropy_batched([t for t, _, _ in ms], 4, 16, seed=7, probe="gaussian",
                                  precision="bf16", power_iters=30)
    for i, (t, R, p) in enumerate(ms):
        lam, _ = O.power_method(R, R_.power_start(R.shape[0], 1, 7), 30)
        assert abs(u[i] - min(1.0, lam)) <= 1e-3 * lam, (i, sizes[i], u[i], lam)


@pytest.mark.parametrize("which", ["1", "2"])
def test_stalled_dependency_times_out_and_context_survives(monkeypatch, which):
    """A dependency that can never be met (VNE_BATCH_TEST_STALL: one tile more
    than the matrix has; 1 = recurrence launch, 2 = power launch) ends each
    bounded wait after its 2-s deadline: the batch returns VNE_ERR_TIMEOUT, and
    the next batch on the same handle runs normally."""
    import time
    ms = mats([200, 333, 129], seed0=700)
    ts = [t for t, _, _ in ms]
    monkeypatch.setenv("VNE_BATCH_TEST_STALL", which)
    t0 = time.perf_counter()
    with pytest.raises(vne.VneError) as err:
        vne.entropy_batched(ts, 6, 16, seed=3, probe="gaussian", precision="bf16")
    dt = time.perf_counter() - t0
    assert err.value.status == 6, err.value  # VNE_ERR_TIMEOUT
    assert 1.5 < dt < 60.0
    monkeypatch.delenv("VNE_BATCH_TEST_STALL")
    hc, _, u = vne.entropy_batched(ts, 6, 16, seed=3, probe="gaussian", precision="bf16")
    for i, (t, R, p) in enumerate(ms):
        rc, _ = oracle_H(R, "chebyshev", 6, 16, 3, u[i])
        assert abs(hc[i] - rc) <= 1e-3 * abs(rc), (i, hc[i], rc)


@pytest.mark.parametrize("precision,method,s", [("bf16", "both", 48), ("bf16x3", "chebyshev", 16)])
def test_batches_outside_the_persistent_path_equal_single_calls(precision, method, s):
    """More than 64 step columns (both estimators, s = 48) or a split precision:
    the batch runs the per-matrix kernels on the streams, bit-identical to the
    single calls."""
    ms = mats([200, 96, 333], seed0=800)
    m, seed = 8, 4
    hc, ht, u = vne.entropy_batched([t for t, _, _ in ms], m, s, seed=seed, probe="gaussian",
                                    precision=precision, method=method)
    kw = dict(seed=seed, probe="gaussian", precision=precision)
    for i, (t, R, p) in enumerate(ms):
        if method == "both":
            one = vne.entropy_both(t, m, s, **kw)
            assert (hc[i], ht[i], u[i]) == (one.H_chebyshev, one.H_taylor, one.u), i
        else:
            one = vne.entropy_chebyshev(t, m, s, **kw)
            assert (hc[i], u[i]) == (one.H, one.u), i
