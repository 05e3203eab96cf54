"""Pins of the oracle's subsampler (Sec. 3.1 Subsampler; the seeded draw is
SplitMix64, pinned to its published outputs)."""
import os
from collections import Counter

import numpy as np
import pytest

import oracle
from paper_2505_02692_b300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
G = 0x9E3779B97F4A7C15
M = (1 << 64) - 1


def test_splitmix64_published_outputs():
    want = []
    with open(os.path.join(HERE, "golden", "splitmix64_published.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                want.append(int(line, 16))
    got = [oracle.splitmix64((k * G) & M) for k in range(len(want))]
    assert got == want


def _cells(task, seed=0, n=300):
    w = synth.make_workload(n, 8, 5, 3, 4, 1, 3, "uniform", seed=seed)
    if task == "within":
        return w, oracle.enumerate_cells(w.labels, 0, (1, 2), None)
    return w, oracle.enumerate_cells(w.labels, 0, (1,), 2)


@pytest.mark.parametrize("task", ["within", "across"])
def test_large_caps_change_nothing(task):
    w, cells = _cells(task)
    big = max(max(len(c.A), len(c.B), len(c.X)) for c in cells)
    sub = oracle.subsample_cells(cells, big, 1000, seed=7)
    assert [(c.P, c.Q, c.by, c.across, sorted(c.A), sorted(c.B), sorted(c.X)) for c in sub] == \
           [(c.P, c.Q, c.by, c.across, sorted(c.A), sorted(c.B), sorted(c.X)) for c in cells]


@pytest.mark.parametrize("task", ["within", "across"])
def test_caps_sizes_subsets_and_counts(task):
    w, cells = _cells(task)
    cap = 2
    sub = oracle.subsample_cells(cells, cap, 0, seed=3)
    orig = {(c.P, c.Q, c.by, c.across): c for c in cells}
    for c in sub:
        o = orig[(c.P, c.Q, c.by, c.across)]
        for r, ro in ((c.A, o.A), (c.B, o.B), (c.X, o.X)):
            assert len(r) == min(cap, len(ro)) and set(r) <= set(ro)
        # |C| by brute force over the kept roles
        assert c.count == sum(1 for x in c.X for a in c.A if a != x for _ in c.B) > 0
    # deterministic, and another seed draws other subsets
    again = oracle.subsample_cells(cells, cap, 0, seed=3)
    assert [(c.A, c.B, c.X) for c in again] == [(c.A, c.B, c.X) for c in sub]
    other = oracle.subsample_cells(cells, cap, 0, seed=4)
    assert [(c.A, c.B, c.X) for c in other] != [(c.A, c.B, c.X) for c in sub]


def test_cap_draw_is_uniform():
    """Each of n items of a role is kept with probability cap / n."""
    c = oracle.Cell(0, 1, (0,), None, list(range(10)), list(range(10, 20)), list(range(10)))
    cap, seeds = 3, 3000
    hits = Counter()
    for s in range(seeds):
        (k,) = oracle.subsample_cells([c], cap, 0, seed=s)
        hits.update(k.B)
    p = cap / 10
    sd = np.sqrt(seeds * p * (1 - p))
    for i in range(10, 20):
        assert abs(hits[i] - seeds * p) < 5 * sd, (i, hits[i])


def test_max_x_across():
    w, cells = _cells("across")
    xmax = 2
    sub = oracle.subsample_cells(cells, 0, xmax, seed=5)
    avail, kept = Counter(), Counter()
    for c in cells:
        avail[(c.by, c.P, c.Q, c.across[0])] += 1
    for c in sub:
        kept[(c.by, c.P, c.Q, c.across[0])] += 1
    for k, n in avail.items():
        assert kept[k] == min(xmax, n)
    # kept across_x values are uniform over the available ones
    key = max(avail, key=lambda k: avail[k])
    tally = Counter()
    for s in range(600):
        for c in oracle.subsample_cells([c for c in cells if (c.by, c.P, c.Q, c.across[0]) == key],
                                        0, 1, seed=s):
            tally[c.across[1]] += 1
    assert len(tally) == avail[key]
    exp = 600 / avail[key]
    assert all(abs(v - exp) < 5 * np.sqrt(exp) for v in tally.values()), tally


def test_subsampled_error_end_to_end():
    """abx_error with caps equals the score of the explicitly subsampled cells."""
    w = synth.tiny_within(seed=2, **synth.HARD)
    err, cells, scores, dd = oracle.abx_error(w.feats, w.offsets, w.labels, 0, (1, 2), None,
                                              [(1,), (2,)], max_size_group=3, seed=11)
    full = oracle.enumerate_cells(w.labels, 0, (1, 2), None)
    sub = oracle.subsample_cells(full, 3, 0, seed=11)
    assert [(c.A, c.B, c.X) for c in sub] == [(c.A, c.B, c.X) for c in cells]
    assert all(s[1] == c.count for s, c in zip(scores, cells))
    assert 0.0 < err < 1.0
