"""The allocation-free power method, vne_lambda_max_static, against the
allocating entry point vne_lambda_max, through the C ABI.

vne_lambda_max_static exists for callers that cannot allocate device memory
when they need the largest eigenvalue (an allocator that forbids new
allocations, a plug-in inside an application that owns the memory budget,
a loop that cannot afford cudaMalloc's implicit synchronisation).  Its scratch
is a fixed device array inside the library, shared by every call; so the test
calls it twice in a row and checks both results, and that a size beyond the
array's limit is refused.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

vne = pytest.importorskip("paper_1801_01072_gb300")
from paper_1801_01072_gb300 import _lib  # noqa: E402

RTOL = 1e-10  # the FP64 parity tolerance of the other GPU tests


def _matrix(t, layout):
    m = _lib.VneMatrix()
    if layout == "dense":
        m.n, m.layout, m.n_diags = t.shape[0], _lib.DENSE, 0
    else:
        m.n, m.layout, m.n_diags = t.shape[1], _lib.DIA, t.shape[0]
    m.dtype = _lib.F64 if t.dtype == torch.float64 else _lib.F32
    m.data = t.data_ptr()
    m.ld = t.stride(0)
    m.memory = _lib.MEM_DEVICE
    return m


def _params(prec, iters, trials, seed):
    p = _lib.VneParams()
    p.m, p.s = 1, 1
    p.precision = _lib.PREC[prec]
    p.probe = 0
    p.seed = seed
    p.power_iters = iters
    p.power_trials = trials
    p.u_scale = 1.0
    p.u_override = 0.0
    return p


def _both(t, layout, prec, iters=30, trials=1, seed=7):
    lib = _lib.load()
    h = C.c_void_p()
    assert lib.vne_create(C.byref(h), torch.cuda.current_device()) == 0
    mat = _matrix(t, layout)
    par = _params(prec, iters, trials, seed)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = C.c_double()
    assert lib.vne_lambda_max(h, C.byref(mat), C.byref(par), C.byref(ref), stream) == 0
    lib.vne_destroy(h)
    got = []
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        lam = C.c_double(-1.0)
        assert lib.vne_lambda_max_static(C.byref(mat), C.byref(par), C.byref(lam), stream) == 0
        got.append(lam.value)
    return ref.value, got


def test_static_dense_f64_matches_allocating_entry_point():
    R, p, _ = synth.dense_exp(512, 50.0, seed=1)
    ref, got = _both(torch.as_tensor(R).cuda(), "dense", "f64", trials=3)
    for g in got:
        assert abs(g - ref) <= RTOL * abs(ref)
    assert p.max() / 6 <= got[0] <= p.max() * (1 + 1e-12)


def test_static_dense_f32_matches_allocating_entry_point():
    # same kernels and block counts as vne_lambda_max: the FP32 sums agree too
    R, _, _ = synth.dense_exp(3000, 300.0, seed=2)
    ref, got = _both(torch.as_tensor(R.astype(np.float32)).cuda(), "dense", "f32", trials=2)
    for g in got:
        assert abs(g - ref) <= 1e-6 * abs(ref)


def test_static_banded_f32_matches_allocating_entry_point():
    vals = synth.band_diag_dominant(100_000, half_bw=16, seed=3, dtype=np.float32)
    ref, got = _both(torch.as_tensor(vals).cuda(), "dia", "f32")
    for g in got:
        assert abs(g - ref) <= RTOL * abs(ref)


def test_static_banded_several_trials():
    vals = synth.band_diag_dominant(40_000, half_bw=8, seed=5, dtype=np.float64)
    ref, got = _both(torch.as_tensor(vals).cuda(), "dia", "f64", trials=3)
    for g in got:
        assert abs(g - ref) <= RTOL * abs(ref)


def test_static_allocates_no_device_memory():
    """The property the entry point exists for: after a first call (which
    loads the library's module), further calls leave the device's free
    memory and torch's allocator statistics unchanged."""
    lib = _lib.load()
    R, _, _ = synth.dense_exp(1024, 100.0, seed=4)
    t = torch.as_tensor(R).cuda()
    mat = _matrix(t, "dense")
    par = _params("f64", 30, 2, 9)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    lam = C.c_double()
    assert lib.vne_lambda_max_static(C.byref(mat), C.byref(par), C.byref(lam), stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(5):
        assert lib.vne_lambda_max_static(C.byref(mat), C.byref(par), C.byref(lam), stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == alloc0


def test_static_refuses_sizes_beyond_its_scratch():
    lib = _lib.load()
    n = 200_000  # n * trials above VNE_STATIC_MAX_VECTOR_ELEMS = 131072
    vals = torch.zeros((2, n), dtype=torch.float64, device="cuda")
    mat = _matrix(vals, "dia")
    par = _params("f64", 3, 1, 1)
    lam = C.c_double()
    st = lib.vne_lambda_max_static(C.byref(mat), C.byref(par), C.byref(lam), None)
    assert st == 8  # VNE_ERR_UNSUPPORTED


def test_static_refuses_a_band_without_diagonals():
    # refused on the host, before any launch
    lib = _lib.load()
    vals = torch.zeros((1, 1000), dtype=torch.float64, device="cuda")
    mat = _matrix(vals, "dia")
    par = _params("f64", 3, 1, 1)
    lam = C.c_double()
    for bad in (0, -1):
        mat.n_diags = bad
        st = lib.vne_lambda_max_static(C.byref(mat), C.byref(par), C.byref(lam), None)
        assert st == 1  # VNE_ERR_INVALID_ARG
