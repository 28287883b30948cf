"""Parity of the random-projection estimator (Algorithm alg:EN) on the GPU
with the CPU FP64 oracle, through the C ABI.

Both sides draw the same projection Pi from their own SplitMix64 code.  The
oracle takes the singular values of R Pi by SVD; the GPU takes the square
roots of the eigenvalues of the FP64 Gram matrix (R Pi)^T (R Pi).  That
route keeps the top singular values to full relative accuracy and the rest
to about sqrt(eps) * p~_1 absolute, so tolerances are on H~ (relative) and
on p~_i relative to p~_1:
  FP64 path   H~ 1e-9,  p~ 1e-9 p~_1
  FP32 path   H~ 1e-4,  p~ 1e-4 p~_1   (FP32 products R Pi, FP64 Gram)
  bf16x3      H~ 1e-4,  p~ 1e-4 p~_1   (R Pi on the tensor cores, two bf16 pieces)
  bf16x6      H~ 2e-5,  p~ 2e-5 p~_1   (three pieces, chunked FP32 accumulation)
"""
import numpy as np
import pytest
import torch

import oracle.projection as OP
import synth

pytestmark = pytest.mark.gpu

vne = pytest.importorskip("paper_1801_01072_gb300")
INVALID_ARG, UNSUPPORTED = 1, 8  # vne_status codes

KINDS = ["gaussian", "srht", "countsketch"]
TOL = {"f64": 1e-9, "f32": 1e-4, "bf16x3": 1e-4, "bf16x6": 2e-5}


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def check(got, ref, prec):
    tol = TOL[prec]
    assert abs(got.H - ref["H"]) <= tol * abs(ref["H"]), (got.H, ref["H"])
    err = np.abs(got.p - ref["p"]).max() / ref["p"][0]
    assert err <= tol, f"p~ error {err:.3e}"


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n,s", [(64, 8), (300, 33), (1000, 100), (257, 512)])
def test_sketch_block_matches_oracle(kind, n, s):
    seed = 77
    got = vne.sketch_block(n, s, seed, kind).cpu().numpy()
    ref = OP.sketch(n, s, kind, seed)
    if kind == "gaussian":
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)
    else:
        # same support and signs exactly; magnitudes 1/sqrt(s) (or 1) to rounding
        assert np.array_equal(np.sign(got), np.sign(ref))
        np.testing.assert_allclose(got, ref, rtol=1e-15, atol=0)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n,k,s", [(64, 4, 8), (300, 10, 33), (1000, 24, 100), (777, 40, 160)])
def test_projection_f64_lowrank(kind, n, k, s):
    R, p, _ = synth.dense_lowrank(n, k, tau=k / 4, seed=n + k)
    got = vne.entropy_projection(dev(R), k, s, kind, seed=5, precision="f64")
    check(got, OP.estimate_projection(R, k, s, kind, seed=5), "f64")


@pytest.mark.parametrize("kind", KINDS)
def test_projection_f32_and_f32_storage(kind):
    n, k, s = 600, 16, 64
    R, p, _ = synth.dense_lowrank(n, k, tau=4.0, seed=8)
    ref = OP.estimate_projection(R, k, s, kind, seed=11)
    got = vne.entropy_projection(dev(R), k, s, kind, seed=11, precision="f32")
    check(got, ref, "f32")
    # FP32 storage converted on the device to the FP64 path: the FP32-rounded R
    R32 = R.astype(np.float32)
    got = vne.entropy_projection(dev(R32), k, s, kind, seed=11, precision="f64")
    check(got, OP.estimate_projection(R32.astype(np.float64), k, s, kind, seed=11), "f64")


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n,k,s", [(300, 10, 33), (1000, 24, 100), (600, 16, 64), (129, 8, 250)])
def test_projection_tensor_core_product(prec, kind, n, k, s):
    """R Pi on the tensor cores (plain-product epilogue), ragged n and s."""
    R, p, _ = synth.dense_lowrank(n, k, tau=k / 4, seed=n + k)
    ref = OP.estimate_projection(R, k, s, kind, seed=5)
    got = vne.entropy_projection(dev(R), k, s, kind, seed=5, precision=prec)
    check(got, ref, prec)


def test_projection_full_rank_spectrum():
    # not the rank-k setting of the theorem: parity still holds step by step
    R, p, _ = synth.dense_exp(256, 30.0, seed=3)
    for kind in KINDS:
        got = vne.entropy_projection(dev(R), 48, 96, kind, seed=2, precision="f64")
        check(got, OP.estimate_projection(R, 48, 96, kind, seed=2), "f64")


def test_projection_largest_sketch_uses_global_scratch():
    # s = 512: the Gram matrix (2 MB) no longer fits in shared memory
    n, k, s = 1500, 100, 512
    R, p, _ = synth.dense_lowrank(n, k, tau=20.0, seed=9)
    got = vne.entropy_projection(dev(R), k, s, "gaussian", seed=4, precision="f64")
    check(got, OP.estimate_projection(R, k, s, "gaussian", seed=4), "f64")


@pytest.mark.parametrize("prec", ["f32", "f64", "bf16x3", "bf16x6"])
def test_projection_bench_workload_full_size(prec):
    w = synth.WORKLOADS["lowrank_n8192_k64"]
    R, p, _ = synth.dense_lowrank(w["n"], w["k"], w["tau"], w["seed"])
    ref = OP.estimate_projection(R, w["k"], w["s"], w["sketch"], seed=1)
    got = vne.entropy_projection(dev(R), w["k"], w["s"], w["sketch"], seed=1, precision=prec)
    check(got, ref, prec)
    # Theorem thm:rp in this setting: the estimate is close to the exact entropy
    H = float(-(p * np.log(p)).sum())
    assert abs(got.H - H) / H < 0.05


def test_projection_edge_cases():
    # n = 1: R = [1], p~ = |Pi_00|
    R = np.ones((1, 1))
    for kind in KINDS:
        got = vne.entropy_projection(dev(R), 1, 1, kind, seed=3)
        check(got, OP.estimate_projection(R, 1, 1, kind, seed=3), "f64")
    # k = s = rank, and s = 1
    R, _, _ = synth.dense_lowrank(130, 5, 2.0, seed=1)
    got = vne.entropy_projection(dev(R), 5, 5, "srht", seed=1)
    check(got, OP.estimate_projection(R, 5, 5, "srht", seed=1), "f64")
    got = vne.entropy_projection(dev(R), 1, 1, "gaussian", seed=1)
    check(got, OP.estimate_projection(R, 1, 1, "gaussian", seed=1), "f64")


def test_projection_rank_deficient_and_host_matrix():
    # k above the rank: the extra p~ are round-off of the Gram route
    # (about sqrt(eps) p~_1) and add a few 1e-6 to H~
    n, r, k, s = 200, 6, 12, 40
    R, p, _ = synth.dense_lowrank(n, r, 3.0, seed=4)
    ref = OP.estimate_projection(R, k, s, "gaussian", seed=6)
    got = vne.entropy_projection(dev(R), k, s, "gaussian", seed=6)
    np.testing.assert_allclose(got.p[:r], ref["p"][:r], rtol=1e-9)
    assert np.all(got.p[r:] < 1e-6 * got.p[0])
    assert abs(got.H - ref["H"]) < 5e-5 * ref["H"]
    host = vne.entropy_projection(torch.as_tensor(R), k, s, "gaussian", seed=6)
    assert host.H == got.H and np.array_equal(host.p, got.p)


def test_projection_error_statuses():
    R = dev(np.eye(16) / 16)

    def status(**kw):
        a = dict(k=2, s=4, sketch="gaussian", precision="f64")
        a.update(kw)
        try:
            vne.entropy_projection(R, **a)
        except vne.VneError as e:
            return e.status
        return 0

    assert status(k=5) == INVALID_ARG          # k > s
    assert status(k=0) == INVALID_ARG
    assert status(s=513, k=2) == UNSUPPORTED   # beyond the eigensolver's N
    assert status(krylov_iters=2, s=128, k=2) == UNSUPPORTED   # block above 64
    assert status(krylov_iters=2, s=4, k=9) == INVALID_ARG     # k above q * b
    assert status(precision="bf16") == UNSUPPORTED
    assert status() == 0


# ---------------------------------------------------------------------------
# block Krylov extension: Ritz values on the same subspace as the oracle
# (FP64 tolerance 1e-9 of theta_1 and H; FP32 1e-4)
# ---------------------------------------------------------------------------

def check_krylov(got, ref, tol):
    assert abs(got.H - ref["H"]) <= tol * abs(ref["H"]), (got.H, ref["H"])
    err = np.abs(got.p - ref["theta"]).max() / ref["theta"][0]
    assert err <= tol, f"theta error {err:.3e}"


@pytest.mark.parametrize("kind", KINDS)
def test_krylov_recovers_rank_k_exactly(kind):
    n, r, b, q = 300, 6, 8, 3
    R, p, _ = synth.dense_lowrank(n, r, 2.0, seed=3)
    got = vne.entropy_projection(dev(R), r, b, kind, seed=2, krylov_iters=q)
    np.testing.assert_allclose(got.p, p, rtol=1e-9)
    H = float(-(p * np.log(p)).sum())
    assert abs(got.H - H) <= 1e-9 * H


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16x3", "bf16x6"])
@pytest.mark.parametrize("n,b,q,k", [(256, 16, 3, 24), (500, 32, 2, 40), (129, 8, 4, 20)])
def test_krylov_parity_full_rank(prec, n, b, q, k):
    R, p, _ = synth.dense_exp(n, 30.0, seed=n)
    drop = 1e-12 if prec == "f64" else 1e-6
    ref = OP.estimate_block_krylov(R, k, b, q, "gaussian", seed=4, drop=drop)
    got = vne.entropy_projection(dev(R), k, b, "gaussian", seed=4, precision=prec,
                                 krylov_iters=q)
    check_krylov(got, ref, 1e-9 if prec == "f64" else 1e-4)


@pytest.mark.parametrize("prec", ["f32", "bf16x3", "bf16x6"])
def test_krylov_bench_shape(prec):
    # block 64, 4 iterations, top-64 Ritz values on the n = 8192 rank-64 matrix
    w = synth.WORKLOADS["lowrank_n8192_k64"]
    R, p, _ = synth.dense_lowrank(w["n"], w["k"], w["tau"], w["seed"])
    got = vne.entropy_projection(dev(R), 64, 64, "gaussian", seed=1, precision=prec,
                                 krylov_iters=4)
    # FP32 products: errors of ~1e-5 of theta_1 on the smallest Ritz values
    assert np.abs(got.p - p).max() <= 1e-4 * p[0]
    H = float(-(p * np.log(p)).sum())
    assert abs(got.H - H) <= 1e-4 * H
