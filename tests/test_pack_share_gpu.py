"""Packed rows shared between tasks of one item set.

abx_distances keeps its packing (normalised, quantised features in the
task's item order, with norms and angles) with the items, and a later task
whose items sort identically reuses it instead of packing again.  Every
result must be bit-identical to the same task on freshly loaded items, the
zero-norm flag must reach the second task too, and the objects may be freed
in any order."""
import numpy as np
import pytest

from paper_2505_02692_b300 import synth

from _common import TASKS

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


def _pairs(w, n=4000, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, w.n_items, n)
    y = rng.integers(0, w.n_items, n)
    return x, y


def _fresh(abx, ctx, w, task, mode, prec):
    on, by, across, levels = TASKS[task]
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, mode, prec)
    return items, cells, dist


def _pack_launches(abx):
    return abx.prof_read().get("pack", (0.0, 0))[1]


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8", "fp32_simt"])
@pytest.mark.parametrize("mode", ["dtw", "mean"])
def test_second_task_reuses_packing(abx, ctx, precision, mode):
    w = synth.medium(seed=21, n_items=900, dim=200, n_context=4, n_speaker=4, n_phone=9,
                     **synth.HARD)
    prec = abx.PRECISIONS[precision]
    md = abx.MEAN if mode == "mean" else abx.DTW
    x, y = _pairs(w)
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    abx.prof_reset()
    abx.prof_enable(True)
    got = {}
    for task in ("within", "across"):   # both sort by (context, speaker, phone)
        on, by, across, levels = TASKS[task]
        cells = abx.abx_build_cells(ctx, items, on, by, across)
        dist = abx.abx_distances(ctx, items, cells, md, prec)
        err, st = abx.abx_score(ctx, dist, cells, levels, recheck=True)
        got[task] = (dist.lookup(x, y), err, st.n_triplets)
        dist.free()
        cells.free()
    abx.prof_enable(False)
    assert _pack_launches(abx) == 1
    items.free()
    for task in ("within", "across"):
        it2, c2, d2 = _fresh(abx, ctx, w, task, md, prec)
        want = d2.lookup(x, y)
        err, st = abx.abx_score(ctx, d2, c2, TASKS[task][3], recheck=True)
        for a, b in zip(got[task][0], want):
            assert np.array_equal(a, b, equal_nan=True)
        assert got[task][1] == err or (np.isnan(err) and np.isnan(got[task][1]))
        assert got[task][2] == st.n_triplets
        d2.free()
        c2.free()
        it2.free()


def test_other_order_or_precision_packs_again(abx, ctx):
    w = synth.medium(seed=22, n_items=600, dim=128, n_context=3, n_speaker=3, n_phone=6)
    x, y = _pairs(w, 2000, 1)
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    on = synth.PHONE
    abx.prof_reset()
    abx.prof_enable(True)
    # by speaker only: items sort by (speaker, phone), a different order
    c1 = abx.abx_build_cells(ctx, items, on, (synth.CONTEXT, synth.SPEAKER), None)
    c2 = abx.abx_build_cells(ctx, items, on, (synth.SPEAKER,), None)
    d1 = abx.abx_distances(ctx, items, c1, abx.DTW, abx.FP32)
    d2 = abx.abx_distances(ctx, items, c2, abx.DTW, abx.FP32)
    d3 = abx.abx_distances(ctx, items, c1, abx.DTW, abx.BF16)
    d4 = abx.abx_distances(ctx, items, c1, abx.DTW, abx.BF16)  # same as d3: reused
    for d in (d1, d2, d3, d4):
        d.sync()
    abx.prof_enable(False)
    assert _pack_launches(abx) == 3
    for d, c, prec in ((d2, (synth.SPEAKER,), abx.FP32), (d4, (synth.CONTEXT, synth.SPEAKER),
                                                           abx.BF16)):
        it2 = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
        cf = abx.abx_build_cells(ctx, it2, on, c, None)
        df = abx.abx_distances(ctx, it2, cf, abx.DTW, prec)
        for a, b in zip(d.lookup(x, y), df.lookup(x, y)):
            assert np.array_equal(a, b, equal_nan=True)
        df.free()
        cf.free()
        it2.free()
    # free in an unusual order: items first, then the distances still read
    items.free()
    a1 = d1.lookup(x, y)
    assert np.isfinite(a1[0][a1[3] > 0]).all()
    for d in (d4, d1, d3, d2):
        d.free()
    c1.free()
    c2.free()


def test_zero_norm_flag_reaches_the_second_task(abx, ctx):
    w = synth.medium(seed=23, n_items=80, dim=32, n_context=2, n_speaker=2, n_phone=4)
    w.feats[5] = 0.0
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    for task in ("within", "across"):
        on, by, across, _ = TASKS[task]
        cells = abx.abx_build_cells(ctx, items, on, by, across)
        dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.FP32)
        with pytest.raises(abx.AbxError) as ei:
            dist.sync()
        assert ei.value.code == -2
        dist.free()
        cells.free()
    items.free()
