"""Pins of the oracle's counter-based probe generator (CPU only)."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        seed, *outs = line.split()
        rows.append((int(seed), [int(o, 16) for o in outs]))
    return rows


@pytest.mark.parametrize("seed,outs", _golden_rows())
def test_splitmix64_published_vectors(seed, outs):
    got = rng.splitmix64(seed, np.arange(len(outs), dtype=np.uint64))
    assert [int(x) for x in got] == outs


def test_probe_layout_is_probe_major_counters():
    n, s, seed = 37, 5, 99
    G = rng.rademacher(n, s, seed)
    for j in range(s):
        c = np.arange(j * n, (j + 1) * n, dtype=np.uint64)
        top = rng.splitmix64(seed, c) >> np.uint64(63)
        assert np.array_equal(G[:, j], np.where(top == 0, 1.0, -1.0))


def test_rademacher_law():
    G = rng.rademacher(1000, 1000, 7)
    assert set(np.unique(G)) == {-1.0, 1.0}
    assert abs(G.mean()) < 5e-3  # 5 sigma at 1e6 draws
    # independent columns: the sample correlation of two columns is O(1/sqrt(n))
    assert abs((G[:, 0] * G[:, 1]).mean()) < 0.2


def test_gaussian_law():
    g = rng.gaussian(1000, 1000, 11).ravel()
    assert abs(g.mean()) < 5e-3
    assert abs(g.var() - 1.0) < 1e-2
    assert abs(stats.kurtosis(g, fisher=False) - 3.0) < 3e-2
    assert stats.kstest(g, "norm").pvalue > 1e-3


def test_power_start_differs_from_probes():
    a = rng.power_start(64, 1, 5)[:, 0]
    b = rng.rademacher(64, 1, 5)[:, 0]
    assert set(np.unique(a)) <= {-1.0, 1.0}
    assert not np.array_equal(a, b)
