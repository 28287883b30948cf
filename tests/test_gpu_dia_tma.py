"""Parity of the FP32 banded step fed by bulk copies (row strides S of 32, 64
and 128 columns) with the CPU FP64 oracle, through the C ABI.

The kernel stages row chunks (192 rows at S = 64, 384 at S = 32, 96 at
S = 128) with a halo of the half-bandwidth rounded up to 4, and fills chunks
that reach outside [0, n) with bounds-checked loads; each CTA walks a
contiguous run of chunks through a ring of 2-4 shared-memory stages.  The
grid below covers single-chunk matrices, sizes on both sides of one and two chunks, stored
diagonal counts below the compiled window (D = 6 runs the 9-diagonal kernel,
D = 13 the 17-diagonal one), Chebyshev-only, Taylor-only and both estimators
(S = s or 2s), Rademacher steps 1 and 2 (probes read from the sign bits) and
Gaussian probes.  Tolerance: 2e-5 relative per moment row and on H, as for
the other FP32 banded tests (FP32 products over at most 33 diagonals).
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle import rng

pytestmark = pytest.mark.gpu

vne = pytest.importorskip("paper_1801_01072_gb300")

TOL = 2e-5


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def moments_close(got, ref, rtol):
    got = np.asarray(got)
    ref = np.asarray(ref)
    sc = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-300)
    err = np.abs(got - ref) / sc
    assert err.max() <= rtol, f"max scaled moment error {err.max():.3e} > {rtol}"


def band(n, hb, seed):
    return synth.band_diag_dominant(n, half_bw=min(hb, max(n - 1, 1)), seed=seed,
                                    dtype=np.float32)


def check(vals, method, s, m=6, seed=3, probe="rademacher", R=None):
    """Run `method` on the band (a tensor, or `vals` copied to the device) and
    compare its moments and estimates with the oracle's."""
    n = vals.shape[1]
    Rop = O.Dia(vals.astype(np.float64))
    u = min(1.0, 2.5 / n)
    G = rng.probes(n, s, seed, probe)
    Rt = R if R is not None else torch.as_tensor(np.ascontiguousarray(vals)).cuda()
    kw = dict(seed=seed, probe=probe, u=u, precision="f32", layout="dia", moments=True)
    if method in ("chebyshev", "both"):
        mu = O.chebyshev_moments(Rop, G, u, m)
    if method in ("taylor", "both"):
        tau = O.taylor_terms(Rop, G, u, m)
    if method == "chebyshev":
        r = vne.entropy_chebyshev(Rt, m, s, **kw)
        moments_close(r.moments, mu, TOL)
        assert rel(r.H, O.chebyshev_estimate_from_moments(mu, u)) < TOL
    elif method == "taylor":
        r = vne.entropy_taylor(Rt, m, s, **kw)
        moments_close(r.moments, tau, TOL)
    else:
        r = vne.entropy_both(Rt, m, s, **kw)
        moments_close(r.moments_chebyshev, mu, TOL)
        moments_close(r.moments_taylor, tau, TOL)
        assert rel(r.H_chebyshev, O.chebyshev_estimate_from_moments(mu, u)) < TOL
    return r


# (method, s): S = 32, 64 and 128 columns, one or two estimators
COLUMNS = [("chebyshev", 32), ("both", 16), ("chebyshev", 64), ("both", 32), ("taylor", 64),
           ("chebyshev", 128), ("both", 64)]
SIZES = [(1, 1), (5, 2), (40, 4), (95, 16), (96, 16), (161, 16), (191, 16), (192, 16),
         (193, 16), (300, 5), (385, 16), (1000, 8), (4099, 12), (20011, 16)]


@pytest.mark.parametrize("n,hb", SIZES)
@pytest.mark.parametrize("method,s", COLUMNS)
def test_dia_tma_parity(n, hb, method, s):
    check(band(n, hb, seed=n + hb), method, s)


@pytest.mark.parametrize("method,s", [("chebyshev", 32), ("chebyshev", 64), ("both", 64)])
def test_dia_tma_many_chunks_per_cta(method, s):
    """Several chunks per CTA, so every stage of the ring is reused (on 152
    SMs: 7 chunks per CTA at S = 32, 14 at S = 64, 28 at S = 128)."""
    check(band(400_009, 16, seed=41), method, s, m=5)


@pytest.mark.parametrize("method,s", [("chebyshev", 32), ("both", 16), ("chebyshev", 128)])
def test_dia_tma_gaussian(method, s):
    check(band(3001, 16, seed=11), method, s, probe="gaussian", seed=8)


def test_dia_tma_matches_register_window_kernel(monkeypatch):
    """The two FP32 kernels (VNE_DIA_TMA=0 selects the register-window one)
    agree with each other and with the oracle on the same inputs."""
    vals = band(50_003, 16, seed=7)
    new = check(vals, "both", 32, m=8)
    monkeypatch.setenv("VNE_DIA_TMA", "0")
    old = check(vals, "both", 32, m=8)
    monkeypatch.delenv("VNE_DIA_TMA")
    moments_close(new.moments_chebyshev, old.moments_chebyshev, 2 * TOL)
    moments_close(new.moments_taylor, old.moments_taylor, 2 * TOL)


def test_dia_tma_strided_and_host_bands():
    """A band with ld > n (a column slice of a wider array), one whose
    diagonals do not start on 16-byte boundaries (the register-window kernel
    takes it), and a band in host memory (copied inside the call)."""
    n, hb = 4097, 16
    vals = band(n, hb, seed=21)
    wide = np.zeros((hb + 1, n + 3), dtype=np.float32)  # ld = 4100, a multiple of 4
    wide[:, :n] = vals
    check(vals, "chebyshev", 64, R=torch.as_tensor(wide).cuda()[:, :n])
    shifted = np.zeros((hb + 1, n + 1), dtype=np.float32)  # data starts 4 bytes in
    shifted[:, 1:] = vals
    check(vals, "chebyshev", 64, R=torch.as_tensor(shifted).cuda()[:, 1:])
    check(vals, "both", 32, R=torch.as_tensor(vals))


def test_dia_tma_garbage_past_the_band_end():
    """Entries vals[d][i] with i >= n - d lie outside R and are ignored, even
    when they hold non-finite values."""
    n, hb = 1000, 16
    vals = band(n, hb, seed=31)
    dirty = vals.copy()
    for d in range(1, hb + 1):
        dirty[d, n - d:] = np.nan
    check(vals, "chebyshev", 64, R=torch.as_tensor(dirty).cuda())
