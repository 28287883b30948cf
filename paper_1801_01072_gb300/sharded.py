"""One estimate split across GPUs by probe range.

The Hutchinson estimate is the mean of per-probe quadratic forms (Lemma
thm:trace), and each probe's moments depend only on R, u and that probe.  So
an s-probe estimate splits into contiguous probe ranges, one per rank: every
rank runs the same power method (same seed, so the same u) and the
recurrence on its probes j0 .. j1-1 (vne_params.probe_offset = j0); the
per-probe moments are gathered in probe order by one all-reduce of an
(m+1) x s array that is zero outside each rank's columns (every entry has a
single non-zero contribution, so the sum is exact); and the final
combination runs on the device with the single call's kernel
(vne_combine_moments).  The result equals the single-GPU call's whenever
the per-probe moments do.  The only collective on the data path is that
all-reduce of 8 (m+1) s bytes per estimator.
"""
from __future__ import annotations

import numpy as np

from . import combine_moments, entropy_both, entropy_chebyshev, entropy_taylor


def probe_range(s: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share [j0, j1) of the s probes for `rank` of `world`:
    the first s mod world ranks take one probe more."""
    if s < 1 or world < 1 or not 0 <= rank < world:
        raise ValueError("need s >= 1 and 0 <= rank < world")
    base, extra = divmod(s, world)
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


def gather_probe_moments(local, j0: int, s: int, group=None):
    """All ranks' per-probe moments in probe order: `local` is this rank's
    (m+1) x (j1 - j0) block (or None for an empty range, with m taken from
    the other ranks); returns the (m+1) x s array on every rank."""
    import torch
    import torch.distributed as dist

    rows = torch.tensor([local.shape[0] if local is not None else 0], dtype=torch.int64)
    dev = "cpu" if dist.get_backend(group) == "gloo" else "cuda"
    rows = rows.to(dev)
    dist.all_reduce(rows, op=dist.ReduceOp.MAX, group=group)
    full = torch.zeros((int(rows.item()), s), dtype=torch.float64, device=dev)
    if local is not None and local.shape[1] > 0:
        full[:, j0:j0 + local.shape[1]] = torch.as_tensor(np.asarray(local), dtype=torch.float64)
    dist.all_reduce(full, group=group)
    return full.cpu().numpy()


def entropy_sharded(R, m: int, s: int, method: str = "both", group=None, **kw):
    """The s-probe estimate of `method` ("chebyshev", "taylor" or "both")
    split across the ranks of `group` by probe range; keyword arguments as
    for the single-GPU calls (seed, probe, precision, power_iters, ...).
    Returns (H_chebyshev, H_taylor, u) on every rank (None for an estimator
    not run)."""
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    j0, j1 = probe_range(s, rank, world)
    mc = mt = None
    if j1 > j0:
        if method == "both":
            r = entropy_both(R, m, j1 - j0, moments=True, probe_offset=j0, **kw)
            mc, mt, u = r.moments_chebyshev, r.moments_taylor, r.u
        elif method == "chebyshev":
            r = entropy_chebyshev(R, m, j1 - j0, moments=True, probe_offset=j0, **kw)
            mc, u = r.moments, r.u
        elif method == "taylor":
            r = entropy_taylor(R, m, j1 - j0, moments=True, probe_offset=j0, **kw)
            mt, u = r.moments, r.u
        else:
            raise ValueError(f"unknown method {method!r}")
    else:
        raise ValueError("every rank needs at least one probe (s >= world size)")
    full_c = gather_probe_moments(mc, j0, s, group) if method in ("both", "chebyshev") else None
    full_t = gather_probe_moments(mt, j0, s, group) if method in ("both", "taylor") else None
    device = R.device.index if getattr(R, "is_cuda", False) else 0
    Hc, Ht = combine_moments(m, s, u, full_c, full_t, device=device)
    return Hc, Ht, u
