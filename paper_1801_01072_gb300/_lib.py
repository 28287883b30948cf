"""ctypes view of the C ABI declared in include/vne.h (marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

VNE_OK = 0
STATUS = {
    0: "VNE_OK", 1: "VNE_ERR_INVALID_ARG", 2: "VNE_ERR_NOT_UNIT_TRACE",
    3: "VNE_ERR_BAD_INTERVAL", 4: "VNE_ERR_OOM", 5: "VNE_ERR_CUDA", 6: "VNE_ERR_TIMEOUT",
    7: "VNE_ERR_NONFINITE", 8: "VNE_ERR_UNSUPPORTED",
}
DENSE, DIA, DENSE_UPPER = 0, 1, 2
F64, F32, C128, C64 = 0, 1, 2, 3
PREC = {"f64": 0, "f32": 1, "bf16": 2, "bf16x3": 3, "bf16x6": 4}
PROBE = {"rademacher": 0, "gaussian": 1}
MEM_DEVICE, MEM_HOST = 0, 1


class VneMatrix(C.Structure):
    _fields_ = [("n", C.c_int64), ("layout", C.c_int32), ("dtype", C.c_int32),
                ("data", C.c_void_p), ("ld", C.c_int64), ("n_diags", C.c_int32),
                ("memory", C.c_int32)]


class VneParams(C.Structure):
    _fields_ = [("m", C.c_int32), ("s", C.c_int32), ("probe", C.c_int32),
                ("precision", C.c_int32), ("seed", C.c_uint64), ("power_iters", C.c_int32),
                ("power_trials", C.c_int32), ("u_scale", C.c_double),
                ("u_override", C.c_double), ("check_trace", C.c_int32),
                ("reserved", C.c_int32), ("probe_offset", C.c_int64)]


class VneError(RuntimeError):
    def __init__(self, status: int, what: str, cuda_err: int = 0):
        self.status = status
        self.cuda_error = cuda_err
        msg = f"{what}: {STATUS.get(status, status)}"
        if cuda_err:
            msg += f" (cudaError {cuda_err})"
        super().__init__(msg)


_LIB = None

# (name, restype, argtypes) for every entry point of include/vne.h
_D = C.POINTER(C.c_double)
_H = C.c_void_p
SIGNATURES = [
    ("vne_create", C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    ("vne_destroy", None, [_H]),
    ("vne_entropy_chebyshev", C.c_int,
     [_H, C.POINTER(VneMatrix), C.POINTER(VneParams), _D, _D, _D, C.c_void_p]),
    ("vne_entropy_taylor", C.c_int,
     [_H, C.POINTER(VneMatrix), C.POINTER(VneParams), _D, _D, _D, C.c_void_p]),
    ("vne_batch_queue", C.c_int64,
     [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_int32,
      C.c_void_p]),
    ("vne_entropy_chebyshev_probes", C.c_int,
     [_H, C.POINTER(VneMatrix), C.c_void_p, C.POINTER(VneParams), _D, _D, _D, C.c_void_p]),
    ("vne_entropy_taylor_probes", C.c_int,
     [_H, C.POINTER(VneMatrix), C.c_void_p, C.POINTER(VneParams), _D, _D, _D, C.c_void_p]),
    ("vne_entropy_both", C.c_int,
     [_H, C.POINTER(VneMatrix), C.POINTER(VneParams), _D, _D, _D, _D, _D, C.c_void_p]),
    ("vne_entropy_batched", C.c_int,
     [_H, C.c_void_p, C.c_int32, C.POINTER(VneParams), C.c_int32, C.c_int32, _D, _D, _D,
      C.c_void_p]),
    ("vne_entropy_sequence", C.c_int,
     [_H, C.c_void_p, C.c_int32, C.POINTER(VneParams), C.c_int32, _D, _D, _D, C.c_void_p]),
    ("vne_tc_autotune", C.c_int,
     [_H, C.POINTER(VneMatrix), C.POINTER(VneParams), C.c_int32, C.c_void_p, _D, C.c_void_p]),
    ("vne_tc_shape", C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_void_p]),
    ("vne_combine_moments", C.c_int,
     [_H, C.c_int32, C.c_int32, C.c_double, C.c_void_p, C.c_void_p, _D, _D, C.c_void_p]),
    ("vne_selftest_timeout", C.c_int, [_H, C.c_void_p]),
    ("vne_lambda_max", C.c_int, [_H, C.POINTER(VneMatrix), C.POINTER(VneParams), _D, C.c_void_p]),
    ("vne_lambda_max_static", C.c_int,
     [C.POINTER(VneMatrix), C.POINTER(VneParams), _D, C.c_void_p]),
    ("vne_entropy_projection", C.c_int,
     [_H, C.POINTER(VneMatrix), C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64,
      _D, _D, C.c_void_p]),
    ("vne_entropy_chebyshev_learned", C.c_int,
     [_H, C.POINTER(VneMatrix), C.POINTER(VneParams), C.c_void_p, _D, _D, _D, C.c_void_p]),
    ("vne_spectral_samples", C.c_int,
     [_H, C.c_int32] + [C.c_void_p] * 7 + [C.c_int32, C.c_int32] + [C.c_void_p] * 5
     + [C.c_void_p]),
    ("vne_mlp_forward", C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    ("vne_mlp_gradient", C.c_int,
     [_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, _D, C.c_void_p]),
    ("vne_mlp_train_step", C.c_int,
     [_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_void_p, C.c_void_p,
      C.c_int64, C.c_int32, C.c_int64, C.c_uint64, _D, C.c_void_p]),
    ("vne_sketch_block", C.c_int,
     [_H, C.c_int64, C.c_int32, C.c_int32, C.c_uint64, C.c_void_p, C.c_void_p]),
    ("vne_probe_block", C.c_int,
     [_H, C.c_int64, C.c_int32, C.c_int32, C.c_uint64, C.c_void_p, C.c_void_p]),
    ("vne_profile_enable", C.c_int, [_H, C.c_int32]),
    ("vne_profile_read", C.c_int, [_H, C.c_int32, _D, C.POINTER(C.c_int64)]),
    ("vne_profile_reset", C.c_int, [_H]),
    ("vne_launch_count", C.c_int64, [_H]),
    ("vne_status_string", C.c_char_p, [C.c_int]),
    ("vne_last_cuda_error", C.c_int32, [_H]),
    ("vne_suggest_m", C.c_int32, [C.c_int32, C.c_double, C.c_double, C.c_double]),
]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libvne.so (building it first if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libvne.so is missing: the CUDA library must be built (no fallback)")
    lib = C.CDLL(_build.LIB)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib
