"""GPU parity of the subsampler (Sec. 3.1 Subsampler): per-cell N and |C| and
the collapsed error equal the oracle's on the same seeded draw."""
import numpy as np
import pytest

import oracle
from paper_2505_02692_b300 import synth

from _common import TASKS, cell_table_oracle, cell_table_product

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


@pytest.mark.parametrize("task,cap,xmax,seed", [
    ("within", 3, 0, 1), ("within", 1, 0, 2), ("within", 7, 0, 3),
    ("across", 2, 0, 4), ("across", 0, 2, 5), ("across", 3, 1, 6), ("across", 0, 1, 7),
])
def test_subsampler_matches_oracle(abx, ctx, task, cap, xmax, seed):
    w = synth.medium(seed=9, n_items=1500, dim=128, n_context=3, n_speaker=4, n_phone=6,
                     **synth.HARD)
    on, by, across, levels = TASKS[task]
    err_o, cells_o, scores_o, _ = oracle.abx_error(w.feats, w.offsets, w.labels, on, by, across,
                                                   levels, max_size_group=cap,
                                                   max_x_across=xmax, seed=seed)
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    cells.set_subsampler(cap, xmax, seed)
    dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.FP32)
    keys, num2, cnt = abx.abx_score_cells(ctx, dist, cells, recheck=True)
    assert cell_table_product(keys, num2, cnt) == cell_table_oracle(cells_o, scores_o, len(by))
    err, st = abx.abx_score(ctx, dist, cells, levels, recheck=True)
    assert err == err_o
    assert st.n_triplets == sum(s[1] for s in scores_o)
    full = cells.info.n_triplets
    assert st.n_triplets < full  # the caps took effect


def test_subsampler_bad_args(abx, ctx):
    w = synth.tiny_within(seed=0)
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, *TASKS["within"][:3])
    with pytest.raises(abx.AbxError):
        cells.set_subsampler(-1, 0, 0)
    with pytest.raises(abx.AbxError):
        cells.set_subsampler(100000, 0, 0)
