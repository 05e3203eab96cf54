"""GPU parity of the cosine, Euclidean and symmetrised KL frame distances
(the "etc." of Score's distance names) against the FP64 oracle, in DTW and
mean-pooled mode.  These distances carry no exact-value intervals, so the FP64 recheck
is refused for them and decisions are compared with a near-tie allowance."""
import numpy as np
import pytest

import oracle
from paper_2505_02692_b300 import synth

from _common import TASKS, cell_table_oracle, cell_table_product

pytestmark = pytest.mark.gpu

TOL = {"fp32_simt": (1e-5, 1e-6), "fp32": (1e-5, 1e-6), "bf16": (2e-3, 2e-3)}


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


@pytest.fixture(scope="module")
def work():
    return synth.medium(seed=31, n_items=900, dim=256, n_context=3, n_speaker=3, n_phone=8,
                        **synth.HARD)


@pytest.mark.parametrize("precision", ["fp32_simt", "fp32", "bf16"])
@pytest.mark.parametrize("kind", ["cosine", "euclidean"])
@pytest.mark.parametrize("mode", ["dtw", "mean"])
def test_other_distance_parity(abx, ctx, work, precision, kind, mode):
    w = work
    okind = {"cosine": oracle.COSINE, "euclidean": oracle.EUCLIDEAN}[kind]
    pkind = {"cosine": abx.COSINE, "euclidean": abx.EUCLIDEAN}[kind]
    omode = oracle.MODE_DTW if mode == "dtw" else oracle.MODE_MEAN
    pmode = abx.DTW if mode == "dtw" else abx.MEAN
    rel, floor = TOL[precision]
    for task in ("within", "across"):
        on, by, across, levels = TASKS[task]
        err_o, cells_o, scores_o, dd = oracle.abx_error(w.feats, w.offsets, w.labels, on, by,
                                                        across, levels, omode, kind=okind)
        items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
        cells = abx.abx_build_cells(ctx, items, on, by, across)
        dist = abx.abx_distances(ctx, items, cells, pmode, abx.PRECISIONS[precision],
                                 distance=pkind)
        pairs = np.array(sorted(dd), dtype=np.int64)
        want = np.array([dd[tuple(p)] for p in pairs])
        d, lo, hi, ln = dist.lookup(pairs[:, 0], pairs[:, 1])
        assert np.all(ln > 0)
        bad = np.abs(d - want) > np.maximum(rel * np.abs(want), floor)
        # FP32 may pick a different one of two near-tied DTW paths
        assert bad.mean() <= (1e-3 if precision != "bf16" else 1e-2), (kind, precision,
                                                                         pairs[bad][:4])
        with pytest.raises(abx.AbxError) as e:
            abx.abx_score(ctx, dist, cells, levels, recheck=True)
        assert e.value.code == -5
        keys, num2, cnt = abx.abx_score_cells(ctx, dist, cells, recheck=False)
        got = cell_table_product(keys, num2, cnt)
        ref = cell_table_oracle(cells_o, scores_o, len(by))
        assert set(got) == set(ref)
        assert all(got[k][1] == ref[k][1] for k in ref)      # |C| always exact
        err, _ = abx.abx_score(ctx, dist, cells, levels, recheck=False)
        if precision == "bf16":
            # BF16 storage without a recheck flips near-tie decisions on this
            # deliberately hard data; the error stays close
            assert abs(err - err_o) < 2e-2
        else:
            differ = sum(got[k] != ref[k] for k in ref)
            assert differ <= max(2, 1e-2 * len(ref)), differ
            assert abs(err - err_o) < 5e-3


# ------------------------------------------------------------------ KL

def _positive(w):
    """Frames made positive (exp of the Gaussian frames), so that each frame
    read as a distribution (divided by its sum) has every component > 0."""
    w.feats = np.exp(0.25 * w.feats).astype(np.float32)
    return w


@pytest.mark.parametrize("mode", ["dtw", "mean"])
def test_kl_distance_parity(abx, ctx, mode):
    """Symmetrised KL on the tensor cores (FP32 split).  The FP16 hi/lo split
    holds each of p and ln p to 22 bits (2^-22 relative per product); what is
    left is the FP32 accumulation of one-signed terms of magnitude up to
    |h_i| + |h_j| + 2 d, with |h| <= ln(dim) = 5.3 here.  No interval is
    derived for KL; the bar is an absolute 1e-4 on d."""
    w = _positive(synth.medium(seed=41, n_items=700, dim=200, n_context=3, n_speaker=3,
                               n_phone=8, **synth.HARD))
    omode = oracle.MODE_DTW if mode == "dtw" else oracle.MODE_MEAN
    pmode = abx.DTW if mode == "dtw" else abx.MEAN
    for task in ("within", "across"):
        on, by, across, levels = TASKS[task]
        err_o, cells_o, scores_o, dd = oracle.abx_error(w.feats, w.offsets, w.labels, on, by,
                                                        across, levels, omode, kind=oracle.KL)
        items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
        cells = abx.abx_build_cells(ctx, items, on, by, across)
        dist = abx.abx_distances(ctx, items, cells, pmode, abx.FP32, distance=abx.KL)
        pairs = np.array(sorted(dd), dtype=np.int64)
        want = np.array([dd[tuple(p)] for p in pairs])
        d, lo, hi, ln = dist.lookup(pairs[:, 0], pairs[:, 1])
        assert np.all(ln > 0)
        assert np.max(np.abs(d - want)) <= 1e-4
        assert np.array_equal(lo, d) and np.array_equal(hi, d)   # no intervals
        with pytest.raises(abx.AbxError) as e:
            abx.abx_score(ctx, dist, cells, levels, recheck=True)
        assert e.value.code == -5
        keys, num2, cnt = abx.abx_score_cells(ctx, dist, cells, recheck=False)
        got = cell_table_product(keys, num2, cnt)
        ref = cell_table_oracle(cells_o, scores_o, len(by))
        assert set(got) == set(ref) and all(got[k][1] == ref[k][1] for k in ref)
        assert sum(got[k] != ref[k] for k in ref) <= max(2, 1e-2 * len(ref))
        err, _ = abx.abx_score(ctx, dist, cells, levels, recheck=False)
        assert abs(err - err_o) < 1e-3


def test_kl_rejects_bad_input(abx, ctx):
    w = _positive(synth.medium(seed=42, n_items=60, dim=24, n_context=2, n_speaker=2,
                               n_phone=4))
    on, by, across, _ = TASKS["within"]
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    with pytest.raises(abx.AbxError) as e:    # built for the FP32 split only
        abx.abx_distances(ctx, items, cells, abx.DTW, abx.BF16, distance=abx.KL)
    assert e.value.code == -5
    w.feats[7, 3] = 0.0                       # a component that is not > 0
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.FP32, distance=abx.KL)
    with pytest.raises(abx.AbxError) as e:
        dist.sync()
    assert e.value.code == -1
