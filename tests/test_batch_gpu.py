"""Batched tasks (abx_batch_*): many ABX tasks of mixed dimensions in shared
launches, replayed from one CUDA graph.

Every task's error must be identical to the one abx_distances + abx_score
give for that task alone (same cells, same decisions, same FP64 summation
order), and, on small tasks, to the FP64 oracle's."""
import numpy as np
import pytest

from paper_2505_02692_b300 import synth

from _common import TASKS, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_02692_b300 import abx as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def ctx(abx):
    return abx.Context(0)


def _tasks(seed=0):
    """Ragged tasks: dims from {200, 256, 512, 768} (200 exercises padding),
    150-600 items, lengths 3-40 skewed short, 5-12 phones."""
    rng = np.random.default_rng(seed)
    dims = [256, 768, 200, 512, 256, 768]
    out = []
    for k, dim in enumerate(dims):
        n = int(rng.integers(150, 600))
        w = synth.make_workload(n, dim, int(rng.integers(5, 13)), 4, 3, 3, 40, "skewed",
                                seed=100 + k, name=f"batch-task-{k}", **synth.HARD)
        out.append(w)
    return out


def _alone(abx, ctx, w, task, mode, precision, recheck=True, weighted=False):
    on, by, across, levels = TASKS[task]
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, mode, precision)
    err, st = abx.abx_score(ctx, dist, cells, levels, weighted=weighted, recheck=recheck)
    return err, st.n_triplets


def _batch(abx, ctx, ws, task, mode, precision, tune=False, recheck=True, weighted=False):
    on, by, across, levels = TASKS[task]
    b = abx.abx_batch_create(ctx, [(w.feats, w.offsets, w.labels) for w in ws], on, by, across,
                             mode, precision, levels, weighted=weighted, recheck=recheck,
                             tune=tune)
    return b


@pytest.mark.parametrize("task", ["within", "across"])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batch_equals_tasks_alone(abx, ctx, task, precision):
    ws = _tasks()
    prec = abx.PRECISIONS[precision]
    b = _batch(abx, ctx, ws, task, abx.DTW, prec)
    assert b.info.n_classes == 4
    b.run()
    err, trip, st = b.wait()
    for k, w in enumerate(ws):
        e1, t1 = _alone(abx, ctx, w, task, abx.DTW, prec)
        assert trip[k] == t1, (k, trip[k], t1)
        assert err[k] == e1 or (np.isnan(err[k]) and np.isnan(e1)), (k, err[k], e1)
    assert st.n_triplets == trip.sum()
    # graph replay gives the same results
    b.run()
    b.run()
    err2, trip2, _ = b.wait()
    assert np.array_equal(err, err2, equal_nan=True) and np.array_equal(trip, trip2)
    assert b.info.graph_kernels > 0
    b.free()


def test_batch_matches_oracle(abx, ctx):
    ws = _tasks(seed=1)[:3]
    b = _batch(abx, ctx, ws, "within", abx.DTW, abx.FP32)
    b.run()
    err, trip, _ = b.wait()
    for k, w in enumerate(ws):
        err_o, cells_o, scores_o, _ = oracle_run(w, "within")
        assert err[k] == err_o, (k, err[k], err_o)
        assert trip[k] == sum(s[1] for s in scores_o)
    b.free()


def test_batch_mean_mode_and_weighted(abx, ctx):
    ws = _tasks(seed=2)
    for weighted in (False, True):
        b = _batch(abx, ctx, ws, "within", abx.MEAN, abx.FP32, weighted=weighted)
        b.run()
        err, trip, _ = b.wait()
        for k, w in enumerate(ws):
            e1, t1 = _alone(abx, ctx, w, "within", abx.MEAN, abx.FP32, weighted=weighted)
            assert err[k] == e1 and trip[k] == t1, (weighted, k, err[k], e1)
        b.free()


def test_batch_tuned_and_eager(abx, ctx, monkeypatch):
    """The autotuner's choice (over the unfused tile and DTW kernel variants),
    the fused kernel and the graph-free path change nothing."""
    ws = _tasks(seed=3)
    b0 = _batch(abx, ctx, ws, "within", abx.DTW, abx.FP32)
    b0.run()
    ref, _, _ = b0.wait()
    b0.free()
    monkeypatch.setenv("ABX_FUSE", "1")
    bf = _batch(abx, ctx, ws, "within", abx.DTW, abx.FP32)
    assert all(bf.info.tile_variant[k] == 4 for k in range(bf.info.n_classes))  # fused
    bf.run()
    got_f, _, _ = bf.wait()
    assert np.array_equal(ref, got_f, equal_nan=True)
    bf.free()
    monkeypatch.delenv("ABX_FUSE")
    b1 = _batch(abx, ctx, ws, "within", abx.DTW, abx.FP32, tune=True)
    info = b1.info
    assert all(0 <= info.dtw_variant[k] < 4 and 0 <= info.tile_variant[k] < 4
               for k in range(info.n_classes))
    b1.run()
    got, _, _ = b1.wait()
    assert np.array_equal(ref, got, equal_nan=True)
    b1.free()
    monkeypatch.setenv("ABX_BATCH_GRAPH", "0")
    b2 = _batch(abx, ctx, ws, "within", abx.DTW, abx.FP32)
    b2.run()
    got2, _, _ = b2.wait()
    assert b2.info.graph_kernels == 0
    assert np.array_equal(ref, got2, equal_nan=True)
    b2.free()


def test_batch_fp8_recheck_exact(abx, ctx):
    """FP8 with interval recheck: every task's error equals the oracle's."""
    ws = _tasks(seed=4)[:2]
    b = _batch(abx, ctx, ws, "within", abx.DTW, abx.FP8)
    b.run()
    err, _, st = b.wait()
    assert st.n_undecided > 0
    for k, w in enumerate(ws):
        err_o, _, _, _ = oracle_run(w, "within")
        assert err[k] == err_o, (k, err[k], err_o)
    b.free()


def test_batch_bad_inputs(abx, ctx):
    w = synth.tiny_within(seed=0)
    on, by, across, levels = TASKS["within"]
    with pytest.raises(abx.AbxError):
        abx.abx_batch_create(ctx, [], on, by, across)
    # collapsing the task attribute is impossible: levels name attributes
    # of the tasks only; an unknown attribute is rejected
    with pytest.raises(abx.AbxError):
        abx.abx_batch_create(ctx, [(w.feats, w.offsets, w.labels)], on, by, across,
                             levels=[(7,)])
