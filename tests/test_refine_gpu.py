"""The refined stage of the recheck (TF32 tensor-core recomputation from the
FP32 features, with a proven interval) against the FP64 oracle.

* abx_refine_pairs: every interval [lo, hi] holds the oracle's DTW distance,
  on the standard and the hard recipe, with items of 1..48 frames (one or
  several passes of up to 16 x 16 frames, one or two 8-column MMA tiles),
  for feature dimensions that are multiples of 16 and of 4 only (the staged
  two-kernel path, with a partial last chunk at 100) and one that is not
  (the fused kernel with scalar loads), for pairs of an item with itself,
  and on adversarial frames whose products are all positive; the intervals
  are narrow (the TF32 rounding angle, not [0, 1]).
* abx_score with the recheck on FP8 and BF16 distances (hard recipe): the
  error equals the oracle's, and the FP64 stage sees at most half of the
  refined pairs.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_02692_b300 import synth

from _common import TASKS, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_02692_b300 import abx as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def ctx(abx):
    return abx.Context(0)


def _workload(seed, n_items, dim, hard, len_hi=48):
    rng = np.random.default_rng(seed)
    lengths = rng.integers(1, len_hi + 1, n_items)
    kw = synth.HARD if hard else {}
    return synth.make_workload(n_items, dim, 6, 3, 3, 1, len_hi, seed=seed, lengths=lengths,
                               name="refine", **kw)


def _check_intervals(abx, ctx, w, px, py, label):
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    lo, hi = abx.abx_refine_pairs(ctx, items, px, py)
    d64, _, _ = oracle.pair_distances(w.feats, w.offsets, px, py)
    inside = (lo <= d64) & (d64 <= hi)
    assert inside.all(), (label, px[~inside][:3], py[~inside][:3], lo[~inside][:3],
                          d64[~inside][:3], hi[~inside][:3])
    width = (hi - lo).astype(np.float64)
    narrow = width < 0.5                 # [0, 1]: nearly parallel frames
    wn = width[narrow] if narrow.any() else np.zeros(1)
    print(f"{label}: {len(px)} pairs, width median {np.median(wn):.2e}, "
          f"q90 {np.quantile(wn, 0.9):.2e}, q99 {np.quantile(wn, 0.99):.2e}, "
          f"max {wn.max():.2e}, {int(np.sum(~narrow))} full")
    return width, narrow


@pytest.mark.parametrize("dim,hard", [(768, False), (768, True), (250, True), (100, True),
                                      (64, False)])
def test_refined_intervals_hold_the_oracle(abx, ctx, dim, hard):
    w = _workload(3 + dim, 400, dim, hard)
    rng = np.random.default_rng(dim)
    n = 3000
    px = rng.integers(0, w.n_items, n)
    py = rng.integers(0, w.n_items, n)
    width, narrow = _check_intervals(abx, ctx, w, px, py, f"dim {dim} hard {hard}")
    # distinct items of random vectors are far from parallel: all narrow.
    # The width is set by the TF32 rounding angle of the frames (2^-11
    # relative per component, about 3e-4 rad as a vector), which moves a
    # frame distance by about 2e-4: widths near 5e-4; a pair whose frames
    # come near |cos| = 0.999 (likelier in 64 dimensions) has a wider
    # interval, where arccos is steep
    other = px != py
    assert narrow[other].all()
    assert np.median(width[other]) < 1e-3
    assert np.quantile(width[other], 0.99) < 3e-3


def test_refined_self_pairs_and_long_items(abx, ctx):
    """d(x, x) = 0 exactly; its frames meet themselves at cos = 1, so the
    interval is [0, 1] (the FP64 stage decides such pairs); the longest
    items need six 8-frame blocks per side."""
    w = _workload(11, 60, 128, False, len_hi=48)
    idx = np.arange(w.n_items)
    width, narrow = _check_intervals(abx, ctx, w, idx, idx, "self pairs")
    longest = np.argsort(-w.lengths)[:10]
    px, py = np.meshgrid(longest, longest)
    keep = px != py
    _check_intervals(abx, ctx, w, px[keep], py[keep], "long items")


def test_refined_intervals_adversarial(abx, ctx):
    """Frames with positive components only (every rounding of the FP32
    sums errs the same way, the worst case of the error model)."""
    rng = np.random.default_rng(21)
    n_items, dim = 120, 768
    lengths = rng.integers(1, 12, n_items)
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    feats = rng.uniform(250.0, 800.0, (int(offsets[-1]), dim)).astype(np.float32)
    mask = rng.random(feats.shape) < 0.5
    feats = np.where(mask, feats * np.float32(0.25), feats).astype(np.float32)
    labels = np.zeros((n_items, 3), dtype=np.int32)
    w = synth.Workload(feats, offsets, labels, 21, "adversarial-refine")
    px, py = np.triu_indices(n_items, 1)
    width, narrow = _check_intervals(abx, ctx, w, px, py, "adversarial")
    assert narrow.all()


def test_refine_pairs_bad_args(abx, ctx):
    w = synth.tiny_within(seed=2)
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    with pytest.raises(abx.AbxError):
        abx.abx_refine_pairs(ctx, items, [0, w.n_items], [1, 0])
    lo, hi = abx.abx_refine_pairs(ctx, items, [], [])
    assert lo.size == 0 and hi.size == 0


@pytest.mark.parametrize("precision", ["fp8", "bf16"])
@pytest.mark.parametrize("task", ["within", "across"])
def test_recheck_stages_exact(abx, ctx, precision, task):
    w = synth.medium(seed=9, n_items=1500, dim=256, n_context=4, n_speaker=4, n_phone=10,
                     **synth.HARD)
    err_o, _, _, _ = oracle_run(w, task)
    on, by, across, levels = TASKS[task]
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.PRECISIONS[precision])
    err, st = abx.abx_score(ctx, dist, cells, levels, recheck=True)
    assert err == err_o, (precision, task, err, err_o)
    assert 0 <= st.n_exact_pairs <= st.n_recheck_pairs
    # the hard recipe crowds the distances, so that the TF32 intervals
    # (about 5e-4 wide) leave a third or so of the refined pairs to FP64;
    # on the standard recipe they settle nearly everything
    if st.n_recheck_pairs > 50:
        assert st.n_exact_pairs < 0.5 * st.n_recheck_pairs
    print(f"{precision} {task}: undecided {st.n_undecided}, refined pairs "
          f"{st.n_recheck_pairs}, FP64 pairs {st.n_exact_pairs}, flips {st.n_flips}")


def test_refine_buffer_overflow_goes_to_fp64(abx, ctx, monkeypatch):
    """With the refined stage's distance buffer capped at 64 KB, most pairs
    do not fit: they keep the interval [0, 1], so their triples must reach
    the FP64 stage, and the error must still be the oracle's."""
    w = synth.medium(seed=9, n_items=1500, dim=256, n_context=4, n_speaker=4, n_phone=10,
                     **synth.HARD)
    err_o, _, _, _ = oracle_run(w, "across")
    on, by, across, levels = TASKS["across"]
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.FP8)
    err_full, st_full = abx.abx_score(ctx, dist, cells, levels, recheck=True)
    monkeypatch.setenv("ABX_REFINE_FD_KB", "64")
    err, st = abx.abx_score(ctx, dist, cells, levels, recheck=True)
    monkeypatch.delenv("ABX_REFINE_FD_KB")
    assert err == err_o and err_full == err_o
    assert st.n_recheck_pairs == st_full.n_recheck_pairs
    assert st.n_exact_pairs > st_full.n_exact_pairs
    print(f"fd buffer 64 KB: FP64 pairs {st.n_exact_pairs} of {st.n_recheck_pairs} "
          f"(full buffer: {st_full.n_exact_pairs})")
