"""The C-ABI library builds, loads and exports every entry point that
include/vne.h declares (CPU only: no compute call needs a GPU here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1801_01072_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(vne_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_estimators():
    names = declared_entry_points()
    for n in ("vne_entropy_chebyshev", "vne_entropy_taylor", "vne_entropy_both",
              "vne_lambda_max", "vne_create", "vne_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert set(declared_entry_points()) <= bound


def test_status_strings(lib):
    for code, name in _lib.STATUS.items():
        assert lib.vne_status_string(code).decode() == name


@pytest.mark.parametrize("method", ["taylor", "chebyshev"])
@pytest.mark.parametrize("u,ell,eps", [(0.5, 0.01, 0.1), (1.0, 1e-3, 0.05), (0.02, 0.019, 0.5)])
def test_suggest_m_matches_oracle(lib, method, u, ell, eps):
    got = lib.vne_suggest_m(0 if method == "taylor" else 1, u, ell, eps)
    assert got == O.suggest_m(method, u, ell, eps)


def test_suggest_m_rejects_bad_arguments(lib):
    assert lib.vne_suggest_m(0, 0.0, 0.1, 0.1) == -1
    assert lib.vne_suggest_m(1, 0.5, 0.6, 0.1) == -1
    assert lib.vne_suggest_m(7, 0.5, 0.1, 0.1) == -1


def test_null_arguments_are_rejected_without_a_gpu(lib):
    # argument checks run before any CUDA call
    H = C.c_double()
    assert lib.vne_entropy_chebyshev(None, None, None, C.byref(H), None, None, None) == 1
    # explicit probes: a NULL probe block is refused first
    assert lib.vne_entropy_chebyshev_probes(None, None, None, None, C.byref(H), None, None,
                                            None) == 1
    assert lib.vne_entropy_taylor_probes(None, None, None, None, C.byref(H), None, None,
                                         None) == 1
    assert lib.vne_create(None, 0) == 1
    assert lib.vne_entropy_sequence(None, None, 1, None, 1, None, None, None, None) == 1


def tc_shape(lib, n, ncols, sms=152):
    out = (C.c_int32 * 4)()
    assert lib.vne_tc_shape(n, ncols, sms, C.cast(out, C.c_void_p)) == 0
    return tuple(out)


@pytest.mark.parametrize("n,ncols,shape", [
    (8192, 256, (256, 1, 1, 2)),   # 64 row tiles: the K split fills 128 SMs in one wave
    (10000, 256, (256, 1, 1, 1)),  # 79 row tiles: a split grid (158 CTAs) would need two waves
    (9728, 256, (256, 1, 1, 2)),   # 76 row tiles: 152 CTAs, exactly one wave
    (9729, 256, (256, 1, 1, 1)),   # 77 row tiles
    (10000, 200, (224, 1, 1, 1)),  # 7 chunks of 32 columns cannot be halved
    (4096, 64, (64, 1, 1, 2)),
    (4096, 32, (32, 1, 1, 1)),     # one chunk: nothing to split
    (2048, 300, (160, 1, 1, 1)),   # two column tiles of 160
    (65536, 256, (256, 1, 1, 1)),  # 512 row tiles fill the GPU without a split
])
def test_tc_shape_rules(lib, n, ncols, shape):
    assert tc_shape(lib, n, ncols) == shape


def test_tc_shape_scales_with_sm_count(lib):
    # the one-wave rule uses the SM count it is given
    assert tc_shape(lib, 8192, 256, sms=100) == (256, 1, 1, 1)
    assert tc_shape(lib, 8192, 256, sms=128) == (256, 1, 1, 2)


def test_tc_shape_rejects_bad_arguments(lib):
    out = (C.c_int32 * 4)()
    assert lib.vne_tc_shape(0, 256, 152, C.cast(out, C.c_void_p)) == 1
    assert lib.vne_tc_shape(8192, 0, 152, C.cast(out, C.c_void_p)) == 1
    assert lib.vne_tc_shape(8192, 256, 0, C.cast(out, C.c_void_p)) == 1
    assert lib.vne_tc_shape(8192, 256, 152, None) == 1
