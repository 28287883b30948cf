"""Learned moment correction of the degree-16 Chebyshev estimator (binding).

The network (19 -> 128 -> 128 -> 128 -> 1, GELU, FP32) maps features of a
Chebyshev estimate of degree 16 -- its probe-total moments tot_k / (s n),
k < 16, and ln(n), ln(lambda~), ln(u) over 10 -- to 100 (H - H_16) / (n u).  Its
training data comes from the library's spectral sampler (probe totals drawn
from a spectrum, labelled by the spectrum's exact entropy); its forward,
backward and Adam passes are the library's kernels.  This module only moves
device pointers and loops over batches.

    from paper_1801_01072_gb300 import learned
    data = learned.spectral_samples(params, m=16, s=128)   # params: per-spectrum draws
    theta = learned.train(theta0, data["features"], data["target"], epochs=20)
    res = learned.entropy_chebyshev_learned(R, theta, s=128, seed=3, precision="bf16")
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib
from . import _handle, _matrix, _params, _stream

N_IN, N_PARAMS, DEGREE = 19, 35713, 16


def _p(t):
    return C.c_void_p(t.data_ptr())


def spectral_samples(spec: dict, m: int = DEGREE, s: int = 128, device: int = 0,
                     totals: bool = False) -> dict:
    """Probe totals, features and labels of the spectra described by `spec`
    (arrays kind, n, a, ktop, floor, c, seed; see vne_spectral_samples)."""
    import torch

    dev = f"cuda:{device}"
    cnt = len(spec["n"])
    t = {k: torch.as_tensor(np.ascontiguousarray(spec[k])).to(dev)
         for k in ("kind", "n", "a", "ktop", "floor", "c")}
    seeds = torch.as_tensor(np.ascontiguousarray(spec["seed"]).view(np.int64)).to(dev)
    out = {"features": torch.empty((cnt, N_IN), dtype=torch.float32, device=dev),
           "target": torch.empty(cnt, dtype=torch.float32, device=dev),
           "H_exact": torch.empty(cnt, dtype=torch.float64, device=dev),
           "H_low": torch.empty(cnt, dtype=torch.float64, device=dev)}
    tot = torch.empty((cnt, m + 1), dtype=torch.float64, device=dev) if totals else None
    h = _handle(device)
    st = h.lib.vne_spectral_samples(
        h.h, cnt, _p(t["kind"]), _p(t["n"]), _p(t["a"]), _p(t["ktop"]), _p(t["floor"]),
        _p(t["c"]), _p(seeds), int(m), int(s), _p(out["features"]), _p(out["target"]),
        _p(out["H_exact"]), _p(out["H_low"]), _p(tot) if tot is not None else None,
        _stream(device, None))
    h.check(st, "vne_spectral_samples")
    if tot is not None:
        out["totals"] = tot
    return out


def mlp_forward(theta, X):
    import torch

    dev = X.device.index
    X = X.contiguous()  # held until the call returns
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    h = _handle(dev)
    h.check(h.lib.vne_mlp_forward(h.h, _p(theta), _p(X), X.shape[0], _p(y),
                                  _stream(dev, None)), "vne_mlp_forward")
    return y


def mlp_gradient(theta, X, target):
    import torch

    dev = X.device.index
    X, target = X.contiguous(), target.contiguous()  # held until the call returns
    g = torch.empty(N_PARAMS, dtype=torch.float32, device=X.device)
    loss = C.c_double()
    h = _handle(dev)
    h.check(h.lib.vne_mlp_gradient(h.h, _p(theta), _p(X), _p(target), X.shape[0], _p(g),
                                   C.byref(loss), _stream(dev, None)), "vne_mlp_gradient")
    return loss.value, g


def train(theta0, X, target, epochs: int = 20, batch: int = 1024, lr: float = 1e-3,
          seed: int = 1, lr_final: float | None = None, report_every: int = 0):
    """Adam on the mean squared error over `epochs` passes of a fixed
    permutation of the rows; the learning rate decays linearly to lr_final
    (default lr / 10).  Returns (theta, list of (step, loss))."""
    import torch

    dev = X.device.index
    theta = theta0.detach().to(torch.float32).contiguous().clone()
    X, target = X.contiguous(), target.contiguous()
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    rows = X.shape[0]
    steps_per_epoch = max(1, rows // batch)
    total = epochs * steps_per_epoch
    lr_final = lr / 10 if lr_final is None else lr_final
    h = _handle(dev)
    stream = _stream(dev, None)
    hist = []
    for step in range(1, total + 1):
        cur = lr + (lr_final - lr) * (step - 1) / max(1, total - 1)
        first = (step - 1) * batch
        loss = C.c_double()
        want = report_every and (step % report_every == 0 or step == total)
        st = h.lib.vne_mlp_train_step(h.h, _p(theta), _p(m), _p(v), step, float(cur), _p(X),
                                      _p(target), rows, batch, first, int(seed),
                                      C.byref(loss) if want else None, stream)
        h.check(st, "vne_mlp_train_step")
        if want:
            hist.append((step, loss.value))
    torch.cuda.synchronize(dev)
    return theta, hist


@dataclass
class LearnedResult:
    H: float          # corrected estimate
    H_plain: float    # the degree-16 estimate it corrects
    u: float


def entropy_chebyshev_learned(R, theta, s: int, seed: int = 0, precision: str = "bf16",
                              m: int = DEGREE, power_iters: int = 30, u_scale: float = 1.05,
                              u: float | None = None, stream=None) -> LearnedResult:
    """Algorithm 1b at degree 16 (Gaussian probes) plus the learned correction."""
    mat, keep, dev = _matrix(R, "dense")
    h = _handle(dev)
    p = _params(m, s, seed, "gaussian", precision, power_iters, 1, u_scale, u, False)
    H, Hp, uo = C.c_double(), C.c_double(), C.c_double()
    st = h.lib.vne_entropy_chebyshev_learned(h.h, C.byref(mat), C.byref(p), _p(theta),
                                             C.byref(H), C.byref(Hp), C.byref(uo),
                                             _stream(dev, stream))
    h.check(st, "vne_entropy_chebyshev_learned")
    del keep
    return LearnedResult(H.value, Hp.value, uo.value)
