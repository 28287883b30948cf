"""Probe-split sharding across ranks (CPU, gloo, world size 2).

The trace estimator is linear in the probes (Lemma thm:trace): splitting the
s probes across ranks, computing each rank's per-probe moments, and summing
the per-degree moment totals with one all-reduce reproduces the single-rank
estimate up to summation order.  This is the exchange a multi-GPU run of one
estimate would need; the benchmark itself shards whole density matrices
across ranks (weak scaling) and needs no data-path collective.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
import synth
from oracle import rng


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, s, m, seed = 96, 10, 12, 5
    R, p, _ = synth.dense_exp(n, 20.0, seed=2)
    u = 1.05 * p.max()
    G = rng.probes(n, s, seed, "gaussian")
    cols = np.array_split(np.arange(s), world)[rank]
    mu = O.chebyshev_moments(R, G[:, cols], u, m).sum(axis=1)      # per-degree totals
    tau = O.taylor_terms(R, G[:, cols], u, m).sum(axis=1)
    t = torch.tensor(np.concatenate([mu, tau]), dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    mu_all, tau_all = t[: m + 1].numpy(), t[m + 1:].numpy()
    a = O.cheb_coefficients(u, m)
    H_cheb = -(a * mu_all).sum() / s
    H_tay = np.log(1 / u) + (tau_all[1:] / np.arange(1, m + 1)).sum() / s
    if rank == 0:
        out.put((H_cheb, H_tay))
    dist.destroy_process_group()


def test_probe_split_allreduce_matches_single_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    H_cheb, H_tay = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    n, s, m, seed = 96, 10, 12, 5
    R, p, _ = synth.dense_exp(n, 20.0, seed=2)
    u = 1.05 * p.max()
    G = rng.probes(n, s, seed, "gaussian")
    ref_c = O.chebyshev_estimate_clenshaw(R, G, u, m)
    ref_t = O.taylor_estimate_from_terms(O.taylor_terms(R, G, u, m), u)
    assert abs(H_cheb - ref_c) < 1e-12 * abs(ref_c)
    assert abs(H_tay - ref_t) < 1e-12 * abs(ref_t)
