"""The context's scratch buffers for the frame-distance tiles.

abx_distances borrows its tile buffer from up to two buffers the context
keeps between calls, in stream order, and allocates one of its own when no
kept buffer is free and large enough.  Calls of different sizes in turn
(a new kept buffer, then none free that fits) and calls from several host
threads on streams of their own (buffers busy, waits across streams) must
give distances, intervals, path lengths and scores bit-identical to a call
on a fresh context, and agree with the FP64 oracle."""
import threading

import numpy as np
import pytest

from paper_2505_02692_b300 import synth

from _common import TASKS, cell_table_oracle, cell_table_product, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_02692_b300 import abx as m
    m.lib()
    return m


def _workloads():
    # three sizes of tile buffer: about 40, 250 and 900 tiles
    return [synth.medium(seed=s, n_items=n, dim=128, n_context=2, n_speaker=4, n_phone=8,
                         **synth.HARD)
            for s, n in ((21, 300), (22, 900), (23, 2000))]


def _dist(abx, ctx, w, task, stream=None):
    on, by, across, levels = TASKS[task]
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.FP32, stream=stream)
    rng = np.random.default_rng(9)
    x = rng.integers(0, w.n_items, 4000)
    y = rng.integers(0, w.n_items, 4000)
    look = dist.lookup(x, y)
    keys, num2, cnt = abx.abx_score_cells(ctx, dist, cells, recheck=True)
    out = (look, cell_table_product(keys, num2, cnt))
    dist.free()
    cells.free()
    items.free()
    return out


def _same(a, b):
    (la, ta), (lb, tb) = a, b
    for u, v in zip(la, lb):
        assert np.array_equal(u, v, equal_nan=True)
    assert ta == tb


def test_scratch_sizes_in_turn(abx):
    """Small, larger, largest, then the small again on one context: the kept
    buffers grow, then the largest call allocates its own; every result
    equals a fresh context's, and the cells the oracle's."""
    ws = _workloads()
    fresh = [_dist(abx, abx.Context(0), w, "across") for w in ws]
    ctx = abx.Context(0)
    for k in (0, 1, 2, 0, 2, 1):
        _same(_dist(abx, ctx, ws[k], "across"), fresh[k])
    err_o, cells_o, scores_o, _ = oracle_run(ws[0], "across")
    assert fresh[0][1] == cell_table_oracle(cells_o, scores_o, 1)


def test_scratch_threads_and_streams(abx):
    """Four host threads, each on a stream of its own, call abx_distances on
    one context at the same time (more calls than kept buffers): results
    equal the single-thread ones."""
    import torch
    ws = _workloads()
    want = {(k, t): _dist(abx, abx.Context(0), ws[k], t)
            for k in (1, 2) for t in ("within", "across")}
    ctx = abx.Context(0)
    jobs = [(k, t) for k in (1, 2) for t in ("within", "across")]
    got, errs = {}, []

    def run(job):
        try:
            s = torch.cuda.Stream()
            for _ in range(2):
                got[job] = _dist(abx, ctx, ws[job[0]], job[1], stream=s.cuda_stream)
        except Exception as e:  # noqa: BLE001 - reported below
            errs.append((job, e))

    th = [threading.Thread(target=run, args=(j,)) for j in jobs]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for j in jobs:
        _same(got[j], want[j])
