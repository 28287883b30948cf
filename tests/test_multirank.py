"""Probe-split sharding across ranks (CPU, gloo, world size 2).

One estimate splits into contiguous probe ranges (the library's
`sharded.probe_range`), each rank produces the per-probe moments of its
range in the library's layout ((m+1) x (j1 - j0), probe order; here the
oracle stands in for the GPU call, since this test runs without a GPU), and
`sharded.gather_probe_moments` assembles the full (m+1) x s array on every
rank with one all-reduce.  The gathered array must equal the rank blocks
side by side exactly, and the estimate from it the single-rank estimate
(Lemma thm:trace: the estimate is the mean of per-probe forms).
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
import synth
from oracle import rng
from paper_1801_01072_gb300.sharded import gather_probe_moments, probe_range

N, S, M, SEED = 96, 11, 12, 5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    R, p, _ = synth.dense_exp(N, 20.0, seed=2)
    return R, 1.05 * p.max(), rng.probes(N, S, SEED, "gaussian")


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    R, u, G = _problem()
    j0, j1 = probe_range(S, rank, world)
    mu = O.chebyshev_moments(R, G[:, j0:j1], u, M)
    tau = O.taylor_terms(R, G[:, j0:j1], u, M)
    full_mu = gather_probe_moments(mu, j0, S)
    full_tau = gather_probe_moments(tau, j0, S)
    out.put((rank, j0, j1, mu, tau, full_mu, full_tau))
    dist.destroy_process_group()


def test_probe_range_partitions_the_probes():
    for s in (1, 2, 7, 64, 129):
        for world in (1, 2, 3, 8):
            if world > s:
                continue
            rs = [probe_range(s, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == s
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        probe_range(4, 4, 4)


def test_probe_split_gather_matches_single_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    got.sort(key=lambda t: t[0])
    blocks_mu = np.concatenate([g[3] for g in got], axis=1)
    blocks_tau = np.concatenate([g[4] for g in got], axis=1)
    for g in got:  # every rank holds the same gathered arrays, equal to the blocks
        assert np.array_equal(g[5], blocks_mu) and np.array_equal(g[6], blocks_tau)
    R, u, G = _problem()
    Hc = O.chebyshev_estimate_from_moments(got[0][5], u)
    Ht = O.taylor_estimate_from_terms(got[0][6], u)
    ref_c = O.chebyshev_estimate_clenshaw(R, G, u, M)
    ref_t = O.taylor_estimate_from_terms(O.taylor_terms(R, G, u, M), u)
    assert abs(Hc - ref_c) < 1e-12 * abs(ref_c)
    assert abs(Ht - ref_t) < 1e-12 * abs(ref_t)
