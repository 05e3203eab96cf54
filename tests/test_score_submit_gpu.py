"""abx_score_submit / abx_score_wait: scoring enqueued without a wait.

Several tasks' scores may be in flight at once and waited for in any order;
each result must be bit-identical to abx_score of the same task, and equal
to the oracle's.  The cell arrays are sized from the candidate count of
abx_build_cells (no read-back at score time), which the wait checks against
the device's own count: degenerate tasks (blocks of one item, groups with a
single on value, one across value) exercise that count.  Freeing the
distances or cells of an outstanding job is refused."""
import numpy as np
import pytest

import oracle
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


def _same(a, b):
    return a == b or (np.isnan(a) and np.isnan(b))


def _stats(st):
    return (st.n_cells, st.n_triplets, st.n_undecided, st.n_recheck_pairs, st.n_flips,
            st.num2_total, st.count2_total)


@pytest.mark.parametrize("mode", ["dtw", "mean"])
@pytest.mark.parametrize("recheck", [0, 1, 2])
def test_two_tasks_in_flight_match_abx_score(abx, ctx, mode, recheck):
    w = synth.medium(seed=31, n_items=700, dim=96, n_context=4, n_speaker=4, n_phone=8,
                     **synth.HARD)
    md = abx.MEAN if mode == "mean" else abx.DTW
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    built = {}
    for task in ("within", "across"):
        on, by, across, levels = TASKS[task]
        cells = abx.abx_build_cells(ctx, items, on, by, across)
        built[task] = (cells, abx.abx_distances(ctx, items, cells, md, abx.BF16), levels)
    want = {t: abx.abx_score(ctx, d, c, lv, recheck=recheck, margin=0.05)
            for t, (c, d, lv) in built.items()}
    for weighted in (False, True):
        jobs = {t: abx.abx_score_submit(ctx, d, c, lv, weighted=weighted, recheck=recheck,
                                        margin=0.05)
                for t, (c, d, lv) in built.items()}
        for t in ("across", "within"):  # waited in the other order
            err, st = jobs[t].wait()
            ref = want[t] if not weighted else abx.abx_score(
                ctx, built[t][1], built[t][0], built[t][2], weighted=True, recheck=recheck,
                margin=0.05)
            assert _same(err, ref[0])
            assert _stats(st) == _stats(ref[1])
    for c, d, _ in built.values():
        d.free()
        c.free()
    items.free()


@pytest.mark.parametrize("task", ["within", "across"])
def test_submitted_score_equals_oracle(abx, ctx, task):
    w = synth.medium(seed=32, n_items=500, dim=64, n_context=3, n_speaker=3, n_phone=7,
                     **synth.HARD)
    on, by, across, levels = TASKS[task]
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.FP32)
    err, st = abx.abx_score_submit(ctx, dist, cells, levels, recheck=True).wait()
    want_err, cells_o, _, _ = oracle_run(w, task)
    assert err == want_err
    assert st.n_cells == len(cells_o)
    dist.free()
    cells.free()
    items.free()


def _degenerate(kind):
    """Seeded workloads whose cells stress the candidate count."""
    rng = np.random.default_rng(7)
    if kind == "singletons":       # every (context, speaker, phone) block has one item
        lab = np.array([(p, c, s) for c in range(3) for s in range(3) for p in range(5)],
                       np.int32)
    elif kind == "one_phone_groups":  # some groups hold a single phone: no cell there
        rows = [(p, c, s) for c in range(4) for s in range(3)
                for p in (range(4) if c % 2 else [c]) for _ in range(2)]
        lab = np.array(rows, np.int32)
    elif kind == "one_speaker":    # across-speaker task with one speaker: no cell at all
        lab = np.array([(p, c, 0) for c in range(3) for p in range(4) for _ in range(3)],
                       np.int32)
    else:                          # sparse: random labels, many empty blocks
        lab = np.stack([rng.integers(0, 9, 300), rng.integers(0, 6, 300),
                        rng.integers(0, 5, 300)], 1).astype(np.int32)
    n = lab.shape[0]
    lens = rng.integers(2, 9, n)
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum(lens)
    feats = rng.standard_normal((int(offs[-1]), 32)).astype(np.float32)
    return feats, offs, lab


@pytest.mark.parametrize("kind", ["singletons", "one_phone_groups", "one_speaker", "sparse"])
@pytest.mark.parametrize("task", ["within", "across"])
def test_candidate_count_on_degenerate_tasks(abx, ctx, kind, task):
    feats, offs, lab = _degenerate(kind)
    on, by, across, levels = TASKS[task]
    items = abx.abx_load_items(ctx, feats, offs, lab)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.FP32)
    err, st = abx.abx_score_submit(ctx, dist, cells, levels, recheck=True).wait()
    want_err, cells_o, _, _ = oracle.abx_error(feats, offs, lab, on, by, across, levels,
                                               oracle.MODE_DTW, False)
    assert st.n_cells == len(cells_o)
    if np.isnan(want_err):
        assert np.isnan(err)
    else:
        assert err == want_err
    dist.free()
    cells.free()
    items.free()


def test_free_refused_while_a_job_is_outstanding(abx, ctx):
    w = synth.medium(seed=33, n_items=200, dim=32, n_context=2, n_speaker=2, n_phone=5)
    on, by, across, levels = TASKS["within"]
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.FP32)
    job = abx.abx_score_submit(ctx, dist, cells, levels, recheck=True)
    for obj in (dist, cells):
        with pytest.raises(abx.AbxError) as ei:
            obj.free()
        assert ei.value.code == -6
    err, st = job.wait()
    assert st.n_triplets > 0 and np.isfinite(err)
    with pytest.raises(abx.AbxError):
        job.wait()
    dist.free()
    cells.free()
    items.free()


def test_zero_norm_reported_by_the_wait(abx, ctx):
    w = synth.medium(seed=34, n_items=80, dim=32, n_context=2, n_speaker=2, n_phone=4)
    w.feats[3] = 0.0
    on, by, across, levels = TASKS["within"]
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.FP32)
    job = abx.abx_score_submit(ctx, dist, cells, levels, recheck=False)
    with pytest.raises(abx.AbxError) as ei:
        job.wait()
    assert ei.value.code == -2
    dist.free()
    cells.free()
    items.free()
