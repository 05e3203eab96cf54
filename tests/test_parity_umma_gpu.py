"""GPU parity of the tcgen05 tensor-core distance kernel (FP32 split, BF16,
FP8) against the FP64 oracle.

FP32 split: per-pair distances within the FP32 tolerance.  All precisions:
the oracle distance lies inside the reported interval [lo, hi] for every
pair, and with the FP64 recheck the per-cell integers N, |C| and the
collapsed error are identical to the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2505_02692_b300 import synth

from _common import TASKS, cell_table_oracle, cell_table_product, oracle_run, within_tol

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


def _run(abx, ctx, w, task, precision, mode=0):
    on, by, across, _ = TASKS[task]
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, mode, abx.PRECISIONS[precision])
    return items, cells, dist


def _pairs(dd):
    pairs = np.array(sorted(dd), dtype=np.int64)
    return pairs, np.array([dd[tuple(p)] for p in pairs])


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("task", ["within", "across"])
def test_umma_medium(abx, ctx, precision, task):
    w = synth.medium(seed=4, n_items=1200, dim=256, n_context=4, n_speaker=4, n_phone=10,
                     **synth.HARD)
    err_o, cells_o, scores_o, dd = oracle_run(w, task)
    assert 0.05 < err_o < 0.45
    items, cells, dist = _run(abx, ctx, w, task, precision)
    pairs, want = _pairs(dd)
    d, lo, hi, ln = dist.lookup(pairs[:, 0], pairs[:, 1])
    assert np.all(ln > 0)
    inside = (lo <= want) & (want <= hi)
    assert inside.all(), (precision, pairs[~inside][:4], lo[~inside][:4], want[~inside][:4],
                          hi[~inside][:4])
    if precision == "fp32":
        ok = within_tol(d, want)
        assert ok.all(), (pairs[~ok][:4], d[~ok][:4], want[~ok][:4])
    keys, num2, cnt = abx.abx_score_cells(ctx, dist, cells, recheck=True)
    assert cell_table_product(keys, num2, cnt) == cell_table_oracle(cells_o, scores_o, 1)
    err, st = abx.abx_score(ctx, dist, cells, TASKS[task][3], recheck=True)
    assert err == err_o
    print(f"{precision} {task}: undecided {st.n_undecided} of {st.n_triplets}, "
          f"recheck pairs {st.n_recheck_pairs}, flips {st.n_flips}, "
          f"max |d - d64| {np.max(np.abs(d - want)):.3e}")


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
def test_umma_tiny_and_edges(abx, ctx, precision):
    # config-0 workload plus items of 1 and 128 frames, 200-dim (padded k)
    w = synth.tiny_within(seed=1, **synth.HARD)
    err_o, cells_o, scores_o, dd = oracle_run(w, "within")
    items, cells, dist = _run(abx, ctx, w, "within", precision)
    pairs, want = _pairs(dd)
    d, lo, hi, ln = dist.lookup(pairs[:, 0], pairs[:, 1])
    assert np.all((lo <= want) & (want <= hi))
    err, _ = abx.abx_score(ctx, dist, cells, TASKS["within"][3], recheck=True)
    assert err == err_o
    rng = np.random.default_rng(12)
    n = 50
    lengths = rng.choice([1, 2, 128, 64, 7], n)
    labels = np.stack([rng.integers(0, 3, n), rng.integers(0, 2, n), rng.integers(0, 2, n)], 1)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    feats = rng.standard_normal((int(offs[-1]), 200)).astype(np.float32)
    w2 = synth.Workload(feats, offs, labels.astype(np.int32), 12, "edges")
    for task in ("within", "across"):
        err_o, cells_o, scores_o, dd = oracle_run(w2, task)
        items, cells, dist = _run(abx, ctx, w2, task, precision)
        pairs, want = _pairs(dd)
        d, lo, hi, ln = dist.lookup(pairs[:, 0], pairs[:, 1])
        assert np.all((lo <= want) & (want <= hi))
        err, _ = abx.abx_score(ctx, dist, cells, TASKS[task][3], recheck=True)
        assert err == err_o or (np.isnan(err) and np.isnan(err_o))


@pytest.mark.parametrize("precision,layout", [("fp32", "0"), ("fp32", "1"), ("bf16", "0")])
def test_umma_store_map_both_paths(abx, ctx, precision, layout, monkeypatch):
    """Items of 1-3 frames put about 64 items in a 128-row panel, so a step
    has column panels of at most 64 items (the narrow kernel stores the
    listed blocks by the per-row-item mask) and panels of more (it stores
    every block).  The narrow kernel (FP32 split) in column-major tiles and
    in strips (ABX_TILE_LAYOUT=1), and the wide kernel (BF16, whole tiles),
    against the oracle: every needed pair computed, the oracle value inside
    its interval, FP32 within the per-pair tolerance, cells bit-exact with
    the recheck."""
    monkeypatch.setenv("ABX_TILE_LAYOUT", layout)
    w = synth.make_workload(900, 128, 6, 2, 3, 1, 3, "uniform", seed=11, name="len1-3",
                            **synth.HARD)
    for task in ("within", "across"):
        err_o, cells_o, scores_o, dd = oracle_run(w, task)
        items, cells, dist = _run(abx, ctx, w, task, precision)
        pairs, want = _pairs(dd)
        d, lo, hi, ln = dist.lookup(pairs[:, 0], pairs[:, 1])
        assert np.all(ln > 0), task
        inside = (lo <= want) & (want <= hi)
        assert inside.all(), (task, pairs[~inside][:3])
        if precision == "fp32":
            ok = within_tol(d, want)
            assert ok.all(), (task, pairs[~ok][:3], d[~ok][:3], want[~ok][:3])
        keys, num2, cnt = abx.abx_score_cells(ctx, dist, cells, recheck=True)
        assert cell_table_product(keys, num2, cnt) == cell_table_oracle(cells_o, scores_o, 1)
        err, _ = abx.abx_score(ctx, dist, cells, TASKS[task][3], recheck=True)
        assert err == err_o, task


@pytest.mark.parametrize("precision,variant", [("fp32", "1"), ("fp32", "2"), ("fp32", "4"),
                                               ("bf16", "0"), ("bf16", "2"), ("fp8", "1")])
def test_umma_kernel_variants(abx, ctx, precision, variant, monkeypatch):
    """The tile kernel variants the autotuner or ABX_UMMA_VARIANT can choose
    besides the defaults: the FP32 split with a 2-stage ring, with 8 epilogue
    warps and on 2-CTA clusters (variant 4, work list built for it); the
    narrow kernel with BF16 / FP8 products (listed-block stores) and the wide
    kernel with 8 epilogue warps.  Each against the oracle: every needed
    pair computed, the oracle value inside its interval, FP32 within the
    per-pair tolerance, cells bit-exact with the recheck."""
    monkeypatch.setenv("ABX_UMMA_VARIANT", variant)
    w = synth.medium(seed=8, n_items=900, dim=256, n_context=3, n_speaker=4, n_phone=8,
                     **synth.HARD)
    for task in ("within", "across"):
        err_o, cells_o, scores_o, dd = oracle_run(w, task)
        items, cells, dist = _run(abx, ctx, w, task, precision)
        pairs, want = _pairs(dd)
        d, lo, hi, ln = dist.lookup(pairs[:, 0], pairs[:, 1])
        assert np.all(ln > 0), task
        inside = (lo <= want) & (want <= hi)
        assert inside.all(), (task, pairs[~inside][:3])
        if precision == "fp32":
            ok = within_tol(d, want)
            assert ok.all(), (task, pairs[~ok][:3], d[~ok][:3], want[~ok][:3])
        keys, num2, cnt = abx.abx_score_cells(ctx, dist, cells, recheck=True)
        assert cell_table_product(keys, num2, cnt) == cell_table_oracle(cells_o, scores_o, 1)
        err, _ = abx.abx_score(ctx, dist, cells, TASKS[task][3], recheck=True)
        assert err == err_o, task


def test_umma_matches_simt_tiles(abx, ctx):
    """FP32 split and CUDA-core FP32 give the same needed pairs and nearly the
    same distances (both within FP32 error of the exact values)."""
    w = synth.medium(seed=5, n_items=700, dim=768, n_context=3, n_speaker=3, n_phone=8,
                     **synth.HARD)
    for task in ("within", "across"):
        _, c1, d1 = _run(abx, ctx, w, task, "fp32_simt")
        _, c2, d2 = _run(abx, ctx, w, task, "fp32")
        assert d1.info.n_pairs == d2.info.n_pairs
        assert d1.info.n_frame_pairs == d2.info.n_frame_pairs
        cells_o = oracle.enumerate_cells(w.labels, *TASKS[task][:3])
        pairs = np.array(oracle.needed_pairs(cells_o))
        a = d1.lookup(pairs[:, 0], pairs[:, 1])[0]
        b = d2.lookup(pairs[:, 0], pairs[:, 1])[0]
        assert np.max(np.abs(a - b)) < 2e-6


def test_umma_mean_mode(abx, ctx):
    w = synth.medium(seed=6, n_items=600, dim=128, n_context=3, n_speaker=3, n_phone=8,
                     noise=12.0, spk_scale=3.0)
    for precision in ("fp32", "bf16"):
        for task in ("within", "across"):
            err_o, cells_o, scores_o, dd = oracle_run(w, task, mode=oracle.MODE_MEAN)
            items, cells, dist = _run(abx, ctx, w, task, precision, mode=abx.MEAN)
            pairs, want = _pairs(dd)
            d, lo, hi, ln = dist.lookup(pairs[:, 0], pairs[:, 1])
            assert np.all((lo <= want) & (want <= hi))
            err, _ = abx.abx_score(ctx, dist, cells, TASKS[task][3], recheck=True)
            assert err == err_o


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
def test_fused_and_unfused_match_the_oracle(abx, ctx, precision, monkeypatch):
    """The fused tile + DTW kernel in both forms (ABX_FUSE=1: a thread per
    pair, in place on the shared d tile; ABX_FUSE=2: 8-lane wavefronts over
    strips of 8 rows, the shorter item on the rows; items of up to 40 frames)
    and the tile-buffer + DTW-kernel path (ABX_FUSE=0), each against the FP64
    oracle: every needed pair computed, the oracle value inside every
    interval, FP32 within the per-pair tolerance, N and |C| of every cell
    bit-exact with the recheck.  Items of 1..40 frames exercise one-row and
    one-column blocks, one to five wavefront strips and the longest rows the
    wavefront's row buffers take.  The three paths evaluate the same cell
    updates on the same frame distances, so their distances, intervals and
    lengths are also bit-identical."""
    rng = np.random.default_rng(7)
    w = synth.make_workload(700, 256, 10, 4, 4, 1, 40, "uniform", seed=7, name="len1-40",
                            **synth.HARD)
    assert w.lengths.max() == 40 and w.lengths.min() == 1
    for task in ("within", "across"):
        err_o, cells_o, scores_o, dd = oracle_run(w, task)
        pairs, want = _pairs(dd)
        got = {}
        for fuse in ("1", "2", "0"):
            monkeypatch.setenv("ABX_FUSE", fuse)
            _, cells, dist = _run(abx, ctx, w, task, precision)
            d, lo, hi, ln = dist.lookup(pairs[:, 0], pairs[:, 1])
            assert np.all(ln > 0), (fuse, task)
            inside = (lo <= want) & (want <= hi)
            assert inside.all(), (fuse, task, pairs[~inside][:3])
            if precision == "fp32":
                ok = within_tol(d, want)
                assert ok.all(), (fuse, task, pairs[~ok][:3], d[~ok][:3], want[~ok][:3])
            keys, num2, cnt = abx.abx_score_cells(ctx, dist, cells, recheck=True)
            assert cell_table_product(keys, num2, cnt) == cell_table_oracle(cells_o, scores_o, 1)
            err, _ = abx.abx_score(ctx, dist, cells, TASKS[task][3], recheck=True)
            assert err == err_o, (fuse, task)
            got[fuse] = (d, lo, hi, ln, dist.info.n_pairs)
        for fuse in ("1", "2"):
            for u, v in zip(got[fuse], got["0"]):
                assert np.array_equal(u, v), (fuse, precision, task)
    monkeypatch.delenv("ABX_FUSE", raising=False)


@pytest.mark.parametrize("precision,margin", [("fp32", 1e-4), ("bf16", 2e-2), ("fp8", 1.0)])
def test_margin_recheck_exact(abx, ctx, precision, margin):
    """Stated-margin recheck: triples whose stored margin is below ``margin``
    are re-decided in FP64.  With margin 1 every triple is re-decided (the
    FP64 recheck path alone must then reproduce the oracle); with the smaller
    margins the stored distances' error must stay below margin / 2 on this
    data, which the test checks before comparing the cells."""
    w = synth.medium(seed=4, n_items=1200, dim=256, n_context=4, n_speaker=4, n_phone=10,
                     **synth.HARD)
    err_o, cells_o, scores_o, dd = oracle_run(w, "within")
    items, cells, dist = _run(abx, ctx, w, "within", precision)
    pairs, want = _pairs(dd)
    d, _, _, _ = dist.lookup(pairs[:, 0], pairs[:, 1])
    assert np.max(np.abs(d - want)) < margin / 2
    err, st = abx.abx_score(ctx, dist, cells, TASKS["within"][3], recheck=abx.RECHECK_MARGIN,
                            margin=margin)
    assert err == err_o
    assert st.n_undecided > 0
    if margin >= 1.0:
        assert st.n_undecided == st.n_triplets
    print(f"{precision} margin {margin}: undecided {st.n_undecided} of {st.n_triplets}, "
          f"flips {st.n_flips}")


def test_margin_recheck_bad_args(abx, ctx):
    w = synth.tiny_within(seed=1, **synth.HARD)
    items, cells, dist = _run(abx, ctx, w, "within", "fp32")
    with pytest.raises(abx.AbxError):
        abx.abx_score(ctx, dist, cells, recheck=abx.RECHECK_MARGIN, margin=-1.0)
    with pytest.raises(abx.AbxError):
        abx.abx_score(ctx, dist, cells, recheck=7)
