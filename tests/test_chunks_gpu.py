"""The tile buffer in several chunks.

abx_distances plans tiles in chunks under a tile-buffer budget
(ABX_TILE_BUDGET_MB, 8 GiB by default) and runs pair planning, the tile
kernel and the DTW once per chunk.  With a budget of 1 MiB (16 tiles per
chunk) every distance, interval and path length, and the scores, must be
bit-identical to the single-chunk run, for each tile kernel and both modes."""
import os

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


def _run(abx, ctx, w, task, mode, prec, budget_mb):
    old = os.environ.get("ABX_TILE_BUDGET_MB")
    if budget_mb is None:
        os.environ.pop("ABX_TILE_BUDGET_MB", None)
    else:
        os.environ["ABX_TILE_BUDGET_MB"] = str(budget_mb)
    try:
        on, by, across, levels = TASKS[task]
        items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
        cells = abx.abx_build_cells(ctx, items, on, by, across)
        dist = abx.abx_distances(ctx, items, cells, mode, prec)
        rng = np.random.default_rng(5)
        x = rng.integers(0, w.n_items, 6000)
        y = rng.integers(0, w.n_items, 6000)
        look = dist.lookup(x, y)
        err, st = abx.abx_score(ctx, dist, cells, levels, recheck=True)
        info = dist.info
        out = (look, err, st.n_triplets, st.n_recheck_pairs, info.n_tiles, info.n_pairs)
        dist.free()
        cells.free()
        items.free()
        return out
    finally:
        if old is None:
            os.environ.pop("ABX_TILE_BUDGET_MB", None)
        else:
            os.environ["ABX_TILE_BUDGET_MB"] = old


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8", "fp32_simt"])
@pytest.mark.parametrize("task", ["within", "across"])
def test_chunked_tile_buffer_is_bit_identical(abx, ctx, precision, task):
    w = synth.medium(seed=41, n_items=900, dim=128, n_context=3, n_speaker=4, n_phone=8,
                     **synth.HARD)
    prec = abx.PRECISIONS[precision]
    one = _run(abx, ctx, w, task, abx.DTW, prec, None)
    many = _run(abx, ctx, w, task, abx.DTW, prec, 1)
    assert one[4] > 16  # more than one chunk of 16 tiles
    for a, b in zip(one[0], many[0]):
        assert np.array_equal(a, b, equal_nan=True)
    assert one[1] == many[1] or (np.isnan(one[1]) and np.isnan(many[1]))
    assert one[2:] == many[2:]


def test_chunked_mean_mode(abx, ctx):
    w = synth.medium(seed=42, n_items=3000, dim=64, n_context=2, n_speaker=3, n_phone=10)
    one = _run(abx, ctx, w, "across", abx.MEAN, abx.FP32, None)
    many = _run(abx, ctx, w, "across", abx.MEAN, abx.FP32, 1)
    assert one[4] > 16
    for a, b in zip(one[0], many[0]):
        assert np.array_equal(a, b, equal_nan=True)
    assert one[1:] == many[1:] or (np.isnan(one[1]) and one[2:] == many[2:])
