"""The work queue of the batched persistent recurrence (host logic, CPU only):
every (matrix, step, tile) item appears once, after all tiles of the previous
step of its matrix (the order that keeps the launch deadlock-free), and the
active set of matrices respects the L2 budget."""
import ctypes as C

import numpy as np
import pytest

from paper_1801_01072_gb300 import _lib, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def queue(lib, sizes, m, s, method, l2_mb, min_tiles):
    n = np.asarray(sizes, dtype=np.int64)
    cnt = lib.vne_batch_queue(n.ctypes.data, len(sizes), m, s, method, l2_mb, min_tiles, None)
    assert cnt > 0
    out = np.zeros((cnt, 4), dtype=np.int32)
    assert lib.vne_batch_queue(n.ctypes.data, len(sizes), m, s, method, l2_mb, min_tiles,
                               out.ctypes.data) == cnt
    return out


def tiles(n):
    return (n + 127) // 128


def rbytes(n):
    return 2 * ((n + 127) // 128 * 128) * ((n + 63) // 64 * 64)


@pytest.mark.parametrize("method,T_extra", [(1, 0), (0, 1), (2, 1)])
@pytest.mark.parametrize("l2_mb,min_tiles", [(64.0, 0), (8.0, 0), (64.0, 304), (1.0, 1000)])
def test_queue_complete_and_dependency_ordered(lib, method, T_extra, l2_mb, min_tiles):
    rng = np.random.default_rng(7)
    sizes = np.floor(256 * 16 ** rng.random(40)).astype(int).tolist() + [1, 127, 128, 129]
    m = 6
    q = queue(lib, sizes, m, 16, method, l2_mb, min_tiles)
    T = m + T_extra
    # every item exactly once
    want = {(j, t, i) for j, n in enumerate(sizes) for t in range(1, T + 1)
            for i in range(tiles(n))}
    got = [tuple(r[:3]) for r in q]
    assert len(got) == len(set(got)) == len(want) and set(got) == want
    # dependencies earlier: every tile of (j, t-1) before any tile of (j, t)
    last = {}
    first = {}
    for k, (j, t, i) in enumerate(got):
        last[(j, t)] = k
        first.setdefault((j, t), k)
    for (j, t), k in first.items():
        if t >= 2:
            assert last[(j, t - 1)] < k


def test_queue_active_set_respects_the_budget(lib):
    sizes = [4096, 4096, 3000, 2048, 1024, 700, 512, 300, 256, 4096]
    budget = 48.0
    q = queue(lib, sizes, 5, 32, 1, budget, 0)
    # matrices are admitted in order; the ones with a step in flight at any
    # point of the queue never exceed the budget unless one matrix alone does
    start = {}
    end = {}
    for k, (j, t, i, _) in enumerate(q):
        start.setdefault(j, k)
        end[j] = k
    assert sorted(start, key=start.get) == list(range(len(sizes)))
    for k in range(len(q)):
        active = [j for j in start if start[j] <= k <= end[j]]
        tot = sum(rbytes(sizes[j]) for j in active)
        assert tot <= budget * 2 ** 20 or len(active) == 1


def test_queue_rejects_bad_arguments(lib):
    n = np.asarray([100], dtype=np.int64)
    assert lib.vne_batch_queue(n.ctypes.data, 1, 0, 4, 1, 64.0, 0, None) == -1
    assert lib.vne_batch_queue(n.ctypes.data, 1, 4, 4, 5, 64.0, 0, None) == -1
    assert lib.vne_batch_queue(None, 1, 4, 4, 1, 64.0, 0, None) == -1
    bad = np.asarray([0], dtype=np.int64)
    assert lib.vne_batch_queue(bad.ctypes.data, 1, 4, 4, 1, 64.0, 0, None) == -1
