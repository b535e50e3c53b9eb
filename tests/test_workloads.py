"""Seeded input generators (no method arithmetic): SplitMix64 against its
published outputs, and the shapes of the workloads' candidate sets."""
import json
import os

import numpy as np

from paper_1602_05510_b300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64.json")))


def test_splitmix64_published_outputs():
    assert [int(x) for x in W.splitmix64_stream(0, 3)] == [int(h, 16) for h in GOLD["seed0"]]
    assert [int(x) for x in W.splitmix64_stream(1234567, 3)] == [int(v) for v in GOLD["seed1234567"]]


def test_counter_form_is_the_stream():
    # output k of candidate c is element (c << 32) + k of the sequential stream
    s = W.splitmix64_stream(99, 10)
    assert np.array_equal(W.counter_u64(99, np.zeros(10, np.uint64), np.arange(10)), s)


def test_draw_range_and_balance():
    u = W.splitmix64_stream(5, 200000)
    for m in (2, 3, 10, 29):
        d = W.draw(u, m)
        assert d.min() == 0 and d.max() == m - 1
        cnt = np.bincount(d.astype(np.int64), minlength=m)
        assert abs(cnt / len(u) - 1 / m).max() < 0.01


def test_exhaustive_and_uniform_shapes():
    e = W.exhaustive_levels(10)
    assert e.shape == (1024, 10) and len({tuple(r) for r in e}) == 1024
    u = W.workload_levels("cfg1", 0, 64)
    assert u.shape == (64, 120) and set(np.unique(u)) <= {0, 1, 2}
    assert np.array_equal(W.workload_levels("cfg1", 10, 5), u[10:15])


def test_uneven_batch():
    n, b, off, lv = W.uneven_candidates(2, 0, 400)
    assert n.min() >= 4 and n.max() <= 32 and set(np.unique(b)) <= {512, 1024, 2048}
    assert np.array_equal(np.diff(off), n.astype(np.int64) * (n + 1) * (n + 2) // 6)
    frac = np.bincount(lv, minlength=3) / len(lv)
    assert abs(frac - [0.5, 0.3, 0.2]).max() < 0.02
