"""Sequences of density matrices (Algorithms 1a/1b with alg:power, applied to
each) estimated one after another, with the transfer of each host-resident
matrix overlapped with the previous estimate: the results equal the single
calls' bit for bit, whatever the memory (pinned, pageable, device) and layout,
and the oracle's where the single calls are pinned to it."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

vne = pytest.importorskip("paper_1801_01072_gb300")


def dense(sizes, seed0=0):
    return [synth.dense_exp(n, max(4.0, n / 10), seed=seed0 + i)[0] for i, n in enumerate(sizes)]


def single(t, m, s, method, layout="dense", **kw):
    if method == "both":
        one = vne.entropy_both(t, m, s, layout=layout, **kw)
        return one.H_chebyshev, one.H_taylor, one.u
    if method == "chebyshev":
        one = vne.entropy_chebyshev(t, m, s, layout=layout, **kw)
        return one.H, None, one.u
    one = vne.entropy_taylor(t, m, s, layout=layout, **kw)
    return None, one.H, one.u


@pytest.mark.parametrize("precision,method", [("bf16", "both"), ("f64", "chebyshev"),
                                              ("f32", "taylor"), ("bf16x3", "both")])
def test_pinned_sequence_equals_single_calls(precision, method):
    sizes = [300, 2048, 97, 1024, 513, 2500]
    Rs = dense(sizes, seed0=10)
    host = [torch.tensor(R).pin_memory() for R in Rs]
    m, s = 12, 16
    kw = dict(seed=4, probe="gaussian", precision=precision)
    hc, ht, u = vne.entropy_sequence(host, m, s, method=method, **kw)
    for i, R in enumerate(Rs):
        c, t, uu = single(torch.tensor(R).cuda(), m, s, method, **kw)
        assert u[i] == uu, i
        if c is not None:
            assert hc[i] == c, (i, hc[i], c)
        if t is not None:
            assert ht[i] == t, (i, ht[i], t)
    if precision == "f64":
        ref = O.estimate(Rs[0], "chebyshev", m, s, 4, "gaussian", power_iters=30)
        assert abs(hc[0] - ref["H"]) <= 1e-10 * abs(ref["H"])


def test_mixed_memory_and_layouts():
    """Pinned, pageable and device matrices, dense and banded, in one call;
    a lone pageable host matrix uses one slot."""
    Rs = dense([400, 1500], seed0=30)
    band = synth.band_diag_dominant(5000, 16, 0.02, seed=2, dtype=np.float64)
    mats = [torch.tensor(Rs[0]).pin_memory(),            # pinned host
            torch.tensor(band),                          # pageable host, banded
            torch.tensor(Rs[1]).cuda(),                  # device
            torch.tensor(Rs[0])]                         # pageable host
    layouts = ["dense", "dia", "dense", "dense"]
    kw = dict(seed=7, probe="rademacher", precision="f64")
    hc, ht, u = vne.entropy_sequence(mats, 8, 6, method="both", layouts=layouts, **kw)
    for i, (t, lay) in enumerate(zip(mats, layouts)):
        c, tt, uu = single(t.cuda(), 8, 6, "both", layout=lay, **kw)
        assert (hc[i], ht[i], u[i]) == (c, tt, uu), i
    assert (hc[3], ht[3]) == (hc[0], ht[0])  # the same matrix from other memory
    one = vne.entropy_sequence([torch.tensor(Rs[1])], 8, 6, method="both", **kw)[0]
    assert one[0] == hc[2]


def test_slots_grow_and_shrink_between_calls():
    """A later call with larger host matrices regrows the device slots; a
    smaller one reuses them."""
    kw = dict(seed=1, probe="gaussian", precision="bf16", method="chebyshev")
    small = [torch.tensor(R).pin_memory() for R in dense([200, 150, 180], seed0=50)]
    big = [torch.tensor(R).pin_memory() for R in dense([3000, 2100], seed0=60)]
    a = vne.entropy_sequence(small, 10, 8, **kw)[0]
    b = vne.entropy_sequence(big, 10, 8, **kw)[0]
    c = vne.entropy_sequence(small, 10, 8, **kw)[0]
    assert np.array_equal(a, c)
    for i, t in enumerate(big):
        assert b[i] == vne.entropy_chebyshev(t.cuda(), 10, 8, seed=1, probe="gaussian",
                                             precision="bf16").H


def test_invalid_matrix_is_refused_before_any_transfer():
    Rs = dense([256], seed0=70)
    wide = torch.zeros((200, 1000), dtype=torch.float64)  # 199 half-bandwidth: unsupported
    with pytest.raises(vne.VneError):
        vne.entropy_sequence([torch.tensor(Rs[0]), wide], 6, 4, layouts=["dense", "dia"],
                             precision="f64")


def test_failing_matrix_stops_the_sequence():
    """With the trace check on, a matrix of trace 2 fails: the ones before it
    keep their estimates, it and the ones after it get NaN, and the call
    returns that matrix's status."""
    from paper_1801_01072_gb300 import _lib
    Rs = dense([300, 200, 250], seed0=80)
    bad = 2.0 * Rs[1]
    host = [torch.tensor(Rs[0]).pin_memory(), torch.tensor(bad).pin_memory(),
            torch.tensor(Rs[2]).pin_memory()]
    mats = [vne._matrix(t, "dense")[0] for t in host]
    arr = (_lib.VneMatrix * 3)(*mats)
    h = vne._handle(torch.cuda.current_device())
    p = vne._params(8, 6, 3, "gaussian", "f64", 30, 1, 1.0, None, True)
    hc = np.zeros(3)
    uo = np.zeros(3)
    st = h.lib.vne_entropy_sequence(h.h, C.cast(arr, C.c_void_p), 3, C.byref(p), 1,
                                    hc.ctypes.data_as(C.POINTER(C.c_double)), None,
                                    uo.ctypes.data_as(C.POINTER(C.c_double)), None)
    assert _lib.STATUS[st] == "VNE_ERR_NOT_UNIT_TRACE"
    H, u = C.c_double(), C.c_double()
    assert h.lib.vne_entropy_chebyshev(h.h, C.byref(mats[0]), C.byref(p), C.byref(H), None,
                                       C.byref(u), None) == 0
    assert hc[0] == H.value and uo[0] == u.value
    assert np.isnan(hc[1:]).all() and np.isnan(uo[1:]).all()


def poisoned(R):
    """R with NaN below the diagonal: a call that read the lower triangle of
    an upper-layout matrix would return NaN."""
    P = R.copy()
    P[np.tril_indices(R.shape[0], -1)] = np.nan
    return P


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16", "bf16x3"])
@pytest.mark.parametrize("where", ["device", "pinned", "pageable"])
def test_upper_layout_equals_dense(precision, where):
    """layout "upper" uses only the upper triangle; on an exactly symmetric
    R the result is the dense layout's, bit for bit (n spans many 32-row
    mirror tiles with a ragged edge)."""
    for n, dt in ((1000, np.float64), (700, np.float32), (2600, np.float64)):
        R = dense([n], seed0=n)[0].astype(dt)
        P = torch.tensor(poisoned(R))
        P = P.cuda() if where == "device" else (P.pin_memory() if where == "pinned" else P)
        kw = dict(seed=3, probe="gaussian", precision=precision)
        got = single(P, 10, 8, "both", layout="upper", **kw)
        want = single(torch.tensor(R).cuda(), 10, 8, "both", **kw)
        assert got == want, (n, got, want)
        lam = vne.lambda_max(P, precision=precision if precision in ("f64", "f32") else "f64",
                             layout="upper")
        assert lam == vne.lambda_max(torch.tensor(R).cuda(),
                                     precision=precision if precision in ("f64", "f32")
                                     else "f64")


def test_upper_layout_sequence_and_batch():
    Rs = dense([1500, 300, 2049], seed0=90)
    host = [torch.tensor(poisoned(R)).pin_memory() for R in Rs]
    kw = dict(seed=5, probe="gaussian", precision="bf16", method="both")
    hc, ht, u = vne.entropy_sequence(host, 12, 16, layouts=["upper"] * 3, **kw)
    bc, bt, bu = vne.entropy_batched([t.cuda() for t in host], 12, 16, layouts=["upper"] * 3,
                                     **kw)
    for i, R in enumerate(Rs):
        c, t, uu = single(torch.tensor(R).cuda(), 12, 16, "both", seed=5, probe="gaussian",
                          precision="bf16")
        assert (hc[i], ht[i], u[i]) == (c, t, uu), i
    # the batch runs its matrices on the per-matrix path: the same bits
    assert np.array_equal(bc, hc) and np.array_equal(bt, ht)


def test_upper_layout_refused_where_unsupported():
    """The projection and allocation-free calls take no upper layout, nor does
    a complex (Hermitian) R: refused before any work."""
    from paper_1801_01072_gb300 import _lib
    R = torch.tensor(dense([256], seed0=3)[0]).cuda()
    mat = vne._matrix(R, "upper")[0]
    h = vne._handle(torch.cuda.current_device())
    H = C.c_double()
    st = h.lib.vne_entropy_projection(h.h, C.byref(mat), 8, 16, 0, 0, 0, 1, C.byref(H), None, None)
    assert _lib.STATUS[st] == "VNE_ERR_INVALID_ARG"  # a layout the projection does not know
    p = vne._params(1, 1, 0, "rademacher", "f64", 30, 1, 1.0, None, False)
    assert _lib.STATUS[h.lib.vne_lambda_max_static(C.byref(mat), C.byref(p), C.byref(H), None)] \
        == "VNE_ERR_INVALID_ARG"
    Cx = torch.tensor(dense([64], seed0=4)[0]).to(torch.complex128).cuda()
    with pytest.raises(vne.VneError):
        vne.entropy_chebyshev(Cx, 4, 4, layout="upper")
