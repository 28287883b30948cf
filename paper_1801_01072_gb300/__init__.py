"""GB300-native randomized von Neumann entropy estimators.

Python binding of the C ABI in ``include/vne.h``: it only marshals torch
tensors (data pointers, sizes, the current CUDA stream) into the library's
calls.  Every step of the method runs in the library's CUDA kernels; there
is no CPU fallback.

    import paper_1801_01072_gb300 as vne
    res = vne.entropy_chebyshev(R, m=20, s=50, seed=1)          # Algorithm 1b
    res = vne.entropy_taylor(R, m=20, s=50, seed=1)             # Algorithm 1a
    both = vne.entropy_both(R, m=40, s=128, precision="bf16")   # shared passes
    lam = vne.lambda_max(R)                                     # Algorithm alg:power
    pr = vne.entropy_projection(R, k=64, s=256, sketch="gaussian")  # Algorithm alg:EN

``R`` is a dense (n, n) tensor (row-major; complex128/complex64 for a
Hermitian R, Section 4) or, with ``layout="dia"``, the
(D, n) band storage ``vals[d, i] = R[i, i + d]`` of a symmetric banded R.
With ``layout="upper"`` only the upper triangle of a dense real R is used
(mirrored on the device).
It may live on the GPU (device pointer) or in host memory (the call then
copies it itself).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import VneError

__all__ = ["entropy_chebyshev", "entropy_taylor", "entropy_both", "lambda_max", "probe_block",
           "entropy_projection", "sketch_block", "ProjectionResult", "entropy_batched", "autotune",
           "Handle", "Result", "BothResult", "entropy_with_probes", "VneError", "suggest_m", "load", "combine_moments"]


def load():
    return _lib.load()


@dataclass
class Result:
    H: float
    u: float
    moments: np.ndarray | None  # (m+1, s)


@dataclass
class BothResult:
    H_chebyshev: float
    H_taylor: float
    u: float
    moments_chebyshev: np.ndarray | None
    moments_taylor: np.ndarray | None


@dataclass
class ProjectionResult:
    H: float
    p: np.ndarray  # (k,) descending


SKETCH = {"gaussian": 0, "srht": 1, "countsketch": 2}


class Handle:
    """Owns a library handle (and its device workspace) on one device."""

    def __init__(self, device: int = 0):
        self.lib = _lib.load()
        h = C.c_void_p()
        st = self.lib.vne_create(C.byref(h), int(device))
        if st != 0:
            raise VneError(st, "vne_create")
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            self.lib.vne_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st: int, what: str):
        if st != 0:
            raise VneError(st, what, int(self.lib.vne_last_cuda_error(self.h)))

    # profiling of the recurrence kernels (CUDA events inside the library)
    def profile(self, on: bool = True):
        self.check(self.lib.vne_profile_enable(self.h, 1 if on else 0), "vne_profile_enable")
        self.check(self.lib.vne_profile_reset(self.h), "vne_profile_reset")

    def profile_read(self, kind: int):
        ms = C.c_double()
        n = C.c_int64()
        self.check(self.lib.vne_profile_read(self.h, kind, C.byref(ms), C.byref(n)),
                   "vne_profile_read")
        return ms.value, n.value

    def launch_count(self) -> int:
        return int(self.lib.vne_launch_count(self.h))


_HANDLES: dict[int, Handle] = {}


def _handle(device: int) -> Handle:
    h = _HANDLES.get(device)
    if h is None:
        h = Handle(device)
        _HANDLES[device] = h
    return h


def _matrix(R, layout: str):
    import torch

    if not isinstance(R, torch.Tensor):
        R = torch.as_tensor(np.ascontiguousarray(R))
    if R.dim() != 2:
        raise ValueError("R must be 2-D")
    if R.dtype not in (torch.float64, torch.float32, torch.complex128, torch.complex64):
        raise ValueError("R must be float64, float32, complex128 or complex64")
    if R.stride(1) != 1:
        R = R.contiguous()
    mat = _lib.VneMatrix()
    if layout in ("dense", "upper"):
        # "upper": only the upper triangle is read (R taken as exactly symmetric)
        if R.shape[0] != R.shape[1]:
            raise ValueError("dense R must be square")
        mat.n = R.shape[0]
        mat.layout = _lib.DENSE if layout == "dense" else _lib.DENSE_UPPER
        mat.n_diags = 0
    elif layout == "dia":
        mat.n = R.shape[1]
        mat.layout = _lib.DIA
        mat.n_diags = R.shape[0]
    else:
        raise ValueError(layout)
    mat.dtype = {torch.float64: _lib.F64, torch.float32: _lib.F32, torch.complex128: _lib.C128,
                 torch.complex64: _lib.C64}[R.dtype]
    mat.data = R.data_ptr()
    mat.ld = R.stride(0)
    mat.memory = _lib.MEM_DEVICE if R.is_cuda else _lib.MEM_HOST
    device = R.device.index if R.is_cuda else torch.cuda.current_device()
    return mat, R, device


def _params(m, s, seed, probe, precision, power_iters, power_trials, u_scale, u, check_trace,
            probe_offset=0):
    p = _lib.VneParams()
    p.probe_offset = int(probe_offset)
    p.m = int(m)
    p.s = int(s)
    p.probe = _lib.PROBE[probe]
    p.precision = _lib.PREC[precision]
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.power_iters = int(power_iters)
    p.power_trials = int(power_trials)
    p.u_scale = float(u_scale)
    p.u_override = float(u) if u is not None else 0.0
    p.check_trace = 1 if check_trace else 0
    return p


def _stream(device, stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream(device)
    return C.c_void_p(stream.cuda_stream)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _estimate(fn_name, R, m, s, seed, probe, precision, power_iters, power_trials, u_scale,
              u, check_trace, moments, layout, stream, probe_offset=0):
    mat, keep, dev = _matrix(R, layout)
    h = _handle(dev)
    p = _params(m, s, seed, probe, precision, power_iters, power_trials, u_scale, u, check_trace,
                probe_offset)
    H = C.c_double()
    uo = C.c_double()
    mom = np.zeros((m + 1, s), dtype=np.float64) if moments else None
    st = getattr(h.lib, fn_name)(h.h, C.byref(mat), C.byref(p), C.byref(H), _dptr(mom),
                                 C.byref(uo), _stream(dev, stream))
    h.check(st, fn_name)
    del keep
    return Result(H.value, uo.value, mom)


def entropy_chebyshev(R, m: int, s: int, seed: int = 0, probe: str = "rademacher",
                      precision: str = "f64", power_iters: int = 30, power_trials: int = 1,
                      u_scale: float = 1.0, u: float | None = None, check_trace: bool = False,
                      moments: bool = False, layout: str = "dense", stream=None,
                      probe_offset: int = 0) -> Result:
    """Algorithm 1b: -(1/s) sum_j g_j^T f_m(R) g_j (Section 3).  probe_offset j0:
    the probes are j0 .. j0+s-1 of the seed's stream."""
    return _estimate("vne_entropy_chebyshev", R, m, s, seed, probe, precision, power_iters,
                     power_trials, u_scale, u, check_trace, moments, layout, stream,
                     probe_offset)


def entropy_taylor(R, m: int, s: int, seed: int = 0, probe: str = "rademacher",
                   precision: str = "f64", power_iters: int = 30, power_trials: int = 1,
                   u_scale: float = 1.0, u: float | None = None, check_trace: bool = False,
                   moments: bool = False, layout: str = "dense", stream=None,
                   probe_offset: int = 0) -> Result:
    """Algorithm 1a: ln u^-1 + (1/s) sum_j sum_k g_j^T R (I - R/u)^k g_j / k (Section 2)."""
    return _estimate("vne_entropy_taylor", R, m, s, seed, probe, precision, power_iters,
                     power_trials, u_scale, u, check_trace, moments, layout, stream,
                     probe_offset)


def entropy_with_probes(R, G, m: int, method: str = "chebyshev", seed: int = 0,
                        precision: str = "f64", power_iters: int = 30, power_trials: int = 1,
                        u_scale: float = 1.0, u: float | None = None, check_trace: bool = False,
                        moments: bool = False, layout: str = "dense", stream=None) -> Result:
    """Algorithm 1b (method "chebyshev") or 1a ("taylor") on the caller's
    probes: G is a CUDA tensor of shape (n, s) (column j = probe g_j), float64
    for precision "f64", else float32.  seed only seeds the power method."""
    import torch

    if method not in ("chebyshev", "taylor"):
        raise ValueError(method)
    if not (isinstance(G, torch.Tensor) and G.is_cuda and G.dim() == 2):
        raise ValueError("G must be a 2-D CUDA tensor (n, s)")
    want = torch.float64 if precision == "f64" else torch.float32
    if G.dtype != want:
        raise ValueError(f"G must be {want} for precision {precision!r}")
    G = G.contiguous()
    mat, keep, dev = _matrix(R, layout)
    if G.shape[0] != mat.n:
        raise ValueError("G must have one row per row of R")
    s = G.shape[1]
    h = _handle(dev)
    p = _params(m, s, seed, "rademacher", precision, power_iters, power_trials, u_scale, u,
                check_trace)
    H = C.c_double()
    uo = C.c_double()
    mom = np.zeros((m + 1, s), dtype=np.float64) if moments else None
    fn = "vne_entropy_chebyshev_probes" if method == "chebyshev" else "vne_entropy_taylor_probes"
    st = getattr(h.lib, fn)(h.h, C.byref(mat), C.c_void_p(G.data_ptr()), C.byref(p), C.byref(H),
                            _dptr(mom), C.byref(uo), _stream(dev, stream))
    h.check(st, fn)
    del keep
    return Result(H.value, uo.value, mom)


def entropy_both(R, m: int, s: int, seed: int = 0, probe: str = "rademacher",
                 precision: str = "f64", power_iters: int = 30, power_trials: int = 1,
                 u_scale: float = 1.0, u: float | None = None, check_trace: bool = False,
                 moments: bool = False, layout: str = "dense", stream=None,
                 probe_offset: int = 0) -> BothResult:
    """Algorithms 1a and 1b on the same probes and u, sharing every pass over R."""
    mat, keep, dev = _matrix(R, layout)
    h = _handle(dev)
    p = _params(m, s, seed, probe, precision, power_iters, power_trials, u_scale, u, check_trace,
                probe_offset)
    Hc, Ht, uo = C.c_double(), C.c_double(), C.c_double()
    mc = np.zeros((m + 1, s)) if moments else None
    mt = np.zeros((m + 1, s)) if moments else None
    st = h.lib.vne_entropy_both(h.h, C.byref(mat), C.byref(p), C.byref(Hc), C.byref(Ht),
                                _dptr(mc), _dptr(mt), C.byref(uo), _stream(dev, stream))
    h.check(st, "vne_entropy_both")
    del keep
    return BothResult(Hc.value, Ht.value, uo.value, mc, mt)


def combine_moments(m: int, s: int, u: float, moments_chebyshev=None, moments_taylor=None,
                    device: int = 0, stream=None):
    """The final combination of Algorithms 1b / 1a from per-probe moments
    ((m+1) x s, probe order), on the device with the single call's kernel.
    Returns (H_chebyshev, H_taylor), None for an estimator not given."""
    h = _handle(device)
    arrs = []
    for mom in (moments_chebyshev, moments_taylor):
        if mom is None:
            arrs.append(None)
            continue
        a = np.ascontiguousarray(np.asarray(mom, dtype=np.float64))
        if a.shape != (m + 1, s):
            raise ValueError(f"moments must be (m+1, s) = {(m + 1, s)}, got {a.shape}")
        arrs.append(a)
    Hc, Ht = C.c_double(), C.c_double()
    st = h.lib.vne_combine_moments(h.h, int(m), int(s), float(u),
                                   arrs[0].ctypes.data if arrs[0] is not None else None,
                                   arrs[1].ctypes.data if arrs[1] is not None else None,
                                   C.byref(Hc), C.byref(Ht), _stream(device, stream))
    h.check(st, "vne_combine_moments")
    return (Hc.value if arrs[0] is not None else None, Ht.value if arrs[1] is not None else None)


def entropy_batched(Rs, m: int, s: int, seed: int = 0, probe: str = "rademacher",
                    precision: str = "f64", method: str = "chebyshev", use_graph: bool = True,
                    power_iters: int = 30, power_trials: int = 1, u_scale: float = 1.0,
                    u: float | None = None, layouts=None, stream=None):
    """Many density matrices (CUDA tensors, uneven sizes) in one call, run
    concurrently and, with use_graph, replayed from one captured CUDA graph.
    Returns (H_chebyshev, H_taylor, u) as float64 arrays (None for an
    estimator not run)."""
    layouts = layouts or ["dense"] * len(Rs)
    mats, keep, dev = [], [], None
    for R, lay in zip(Rs, layouts):
        mat, k, d = _matrix(R, lay)
        if not R.is_cuda:
            raise ValueError("entropy_batched takes device tensors")
        mats.append(mat)
        keep.append(k)
        dev = d if dev is None else dev
    arr = (_lib.VneMatrix * len(mats))(*mats)
    h = _handle(dev)
    p = _params(m, s, seed, probe, precision, power_iters, power_trials, u_scale, u, False)
    meth = {"taylor": 0, "chebyshev": 1, "both": 2}[method]
    n = len(mats)
    hc = np.full(n, np.nan) if meth in (1, 2) else None
    ht = np.full(n, np.nan) if meth in (0, 2) else None
    uo = np.zeros(n)
    st = h.lib.vne_entropy_batched(h.h, C.cast(arr, C.c_void_p), n, C.byref(p), meth,
                                   1 if use_graph else 0, _dptr(hc), _dptr(ht), _dptr(uo),
                                   _stream(dev, stream))
    h.check(st, "vne_entropy_batched")
    del keep
    return hc, ht, uo


def entropy_sequence(Rs, m: int, s: int, seed: int = 0, probe: str = "rademacher",
                     precision: str = "f64", method: str = "chebyshev", power_iters: int = 30,
                     power_trials: int = 1, u_scale: float = 1.0, u: float | None = None,
                     layouts=None, stream=None):
    """Density matrices (host or device tensors) estimated one after another
    with the single call's kernels; a host matrix's transfer (pinned memory)
    runs while the previous matrix is estimated.  Returns (H_chebyshev,
    H_taylor, u) as float64 arrays (None for an estimator not run)."""
    layouts = layouts or ["dense"] * len(Rs)
    mats, keep, dev, host_dev = [], [], None, None
    for R, lay in zip(Rs, layouts):
        mat, k, d = _matrix(R, lay)
        mats.append(mat)
        keep.append(k)
        if k.is_cuda:
            if dev is not None and d != dev:
                raise ValueError("entropy_sequence takes tensors of one device")
            dev = d
        else:
            host_dev = d
    dev = host_dev if dev is None else dev
    arr = (_lib.VneMatrix * len(mats))(*mats)
    h = _handle(dev)
    p = _params(m, s, seed, probe, precision, power_iters, power_trials, u_scale, u, False)
    meth = {"taylor": 0, "chebyshev": 1, "both": 2}[method]
    n = len(mats)
    hc = np.full(n, np.nan) if meth in (1, 2) else None
    ht = np.full(n, np.nan) if meth in (0, 2) else None
    uo = np.full(n, np.nan)
    st = h.lib.vne_entropy_sequence(h.h, C.cast(arr, C.c_void_p), n, C.byref(p), meth,
                                    _dptr(hc), _dptr(ht), _dptr(uo), _stream(dev, stream))
    h.check(st, "vne_entropy_sequence")
    del keep
    return hc, ht, uo


def autotune(R, m: int, s: int, precision: str = "bf16", method: str = "chebyshev",
             seed: int = 0, probe: str = "gaussian", power_iters: int = 30, stream=None):
    """Time the tensor-core tile shapes on R and keep the fastest for R's size
    bucket.  Returns ((BN, CM, CN, ksplit), microseconds per step)."""
    mat, keep, dev = _matrix(R, "dense")
    h = _handle(dev)
    p = _params(m, s, seed, probe, precision, power_iters, 1, 1.0, None, False)
    shape = (C.c_int32 * 4)()
    us = C.c_double()
    meth = {"taylor": 0, "chebyshev": 1, "both": 2}[method]
    st = h.lib.vne_tc_autotune(h.h, C.byref(mat), C.byref(p), meth, C.cast(shape, C.c_void_p),
                               C.byref(us), _stream(dev, stream))
    h.check(st, "vne_tc_autotune")
    del keep
    return tuple(shape), us.value


def lambda_max(R, power_iters: int = 30, power_trials: int = 1, seed: int = 0,
               precision: str = "f64", u_scale: float = 1.0, layout: str = "dense",
               stream=None) -> float:
    """Algorithm alg:power: max over trials of the Rayleigh quotient of R^t x_0."""
    mat, keep, dev = _matrix(R, layout)
    h = _handle(dev)
    p = _params(1, 1, seed, "rademacher", precision, power_iters, power_trials, u_scale, None,
                False)
    lam = C.c_double()
    st = h.lib.vne_lambda_max(h.h, C.byref(mat), C.byref(p), C.byref(lam), _stream(dev, stream))
    h.check(st, "vne_lambda_max")
    del keep
    return lam.value


def probe_block(n: int, s: int, seed: int, probe: str = "rademacher", device: int = 0):
    """The library's probe block as a (n, s) float64 CUDA tensor (column j = g_j)."""
    import torch

    h = _handle(device)
    out = torch.empty((s, n), dtype=torch.float64, device=f"cuda:{device}")
    st = h.lib.vne_probe_block(h.h, int(n), int(s), _lib.PROBE[probe], int(seed),
                               C.c_void_p(out.data_ptr()), _stream(device, None))
    h.check(st, "vne_probe_block")
    return out.t()


def entropy_projection(R, k: int, s: int, sketch: str = "gaussian", seed: int = 0,
                       precision: str = "f64", krylov_iters: int = 0,
                       stream=None) -> ProjectionResult:
    """Algorithm alg:EN: the k largest singular values p~ of R Pi and sum p~ ln(1/p~)."""
    mat, keep, dev = _matrix(R, "dense")
    h = _handle(dev)
    H = C.c_double()
    p = np.zeros(int(k), dtype=np.float64)
    st = h.lib.vne_entropy_projection(h.h, C.byref(mat), int(k), int(s), SKETCH[sketch],
                                      int(krylov_iters), _lib.PREC[precision],
                                      int(seed) & 0xFFFFFFFFFFFFFFFF, C.byref(H), _dptr(p),
                                      _stream(dev, stream))
    h.check(st, "vne_entropy_projection")
    del keep
    return ProjectionResult(H.value, p)


def sketch_block(n: int, s: int, seed: int, sketch: str = "gaussian", device: int = 0):
    """The random projection Pi as a (n, s) float64 CUDA tensor."""
    import torch

    h = _handle(device)
    out = torch.empty((s, n), dtype=torch.float64, device=f"cuda:{device}")
    st = h.lib.vne_sketch_block(h.h, int(n), int(s), SKETCH[sketch], int(seed),
                                C.c_void_p(out.data_ptr()), _stream(device, None))
    h.check(st, "vne_sketch_block")
    return out.t()


def suggest_m(method: str, u: float, ell: float, eps: float) -> int:
    lib = _lib.load()
    return int(lib.vne_suggest_m(0 if method == "taylor" else 1, u, ell, eps))
