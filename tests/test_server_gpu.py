"""Serving loop (abx_server_*): jobs that arrive while others run are admitted
into new batches; every job's result must be the same alone and in the mix
(identical errors: the batches reproduce the single-task computation)."""
import time

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


def _jobs(seed=0, n_dumps=3, layers=3):
    """Dumps of a few layers each: a dump's layers share items and labels and
    differ in features (another seed); dims and sizes vary across dumps."""
    rng = np.random.default_rng(seed)
    jobs = []
    for d in range(n_dumps):
        n = int(rng.integers(150, 500))
        dim = int(rng.choice([200, 256, 512]))
        base = synth.make_workload(n, dim, 8, 4, 3, 3, 25, "skewed", seed=10 * d + 1,
                                   name=f"dump{d}", **synth.HARD)
        for layer in range(layers):
            w = synth.make_workload(n, dim, 8, 4, 3, 3, 25, "skewed", seed=10 * d + 1,
                                    name=f"dump{d}-l{layer}", lengths=base.lengths,
                                    **synth.HARD)
            # same items and labels, other frames for each layer
            feats = w.feats + np.float32(0.5 * layer) * np.random.default_rng(layer).standard_normal(
                w.feats.shape, dtype=np.float32)
            jobs.append((np.ascontiguousarray(feats), base.offsets, base.labels))
    return jobs


def _alone(abx, ctx, job, precision):
    feats, offs, labels = job
    items = abx.abx_load_items(ctx, feats, offs, labels)
    out = []
    for task in ("within", "across"):
        on, by, across, levels = TASKS[task]
        cells = abx.abx_build_cells(ctx, items, on, by, across)
        dist = abx.abx_distances(ctx, items, cells, abx.DTW, precision)
        err, st = abx.abx_score(ctx, dist, cells, levels, recheck=True)
        out.append((err, st.n_triplets))
    return out


def _specs(abx):
    return [abx.task_spec(*TASKS[t]) for t in ("within", "across")]


def test_server_mix_equals_alone(abx):
    jobs = _jobs()
    ctx_alone = abx.Context(0)
    ref = [_alone(abx, ctx_alone, j, abx.BF16) for j in jobs]
    ctx = abx.Context(0)
    srv = abx.Server(ctx, 3, _specs(abx), abx.DTW, abx.BF16, recheck=True, max_inflight=2,
                     max_batch_jobs=4)
    # half at once, the rest staggered so they arrive while batches run
    tickets = [srv.submit(*j) for j in jobs[:4]]
    for j in jobs[4:]:
        time.sleep(0.01)
        tickets.append(srv.submit(*j))
    res = [srv.wait(t) for t in tickets]
    st = srv.stats
    srv.close()
    assert st.completed == len(jobs) and st.failed == 0
    assert st.batches < len(jobs)  # some jobs shared a batch
    for k, r in enumerate(res):
        assert r.status == 0
        assert r.t_submit <= r.t_admit <= r.t_launch <= r.t_done
        for q in range(2):
            e, t = ref[k][q]
            assert r.errors[q] == e or (np.isnan(r.errors[q]) and np.isnan(e)), (k, q)
            assert r.triplets[q] == t


def test_server_budget_one_at_a_time(abx):
    """A budget smaller than any job: jobs still run, one batch each."""
    jobs = _jobs(seed=1, n_dumps=2, layers=2)
    ctx = abx.Context(0)
    srv = abx.Server(ctx, 3, _specs(abx), abx.DTW, abx.FP32, recheck=True, hbm_budget=1)
    tickets = [srv.submit(*j) for j in jobs]
    res = [srv.wait(t) for t in tickets]
    st = srv.stats
    srv.close()
    assert all(r.status == 0 for r in res)
    assert st.batches == len(jobs)
    assert len({r.batch_id for r in res}) == len(jobs)


def test_server_poll_and_bad_input(abx):
    jobs = _jobs(seed=2, n_dumps=1, layers=1)
    ctx = abx.Context(0)
    srv = abx.Server(ctx, 3, _specs(abx), abx.DTW, abx.FP32)
    t = srv.submit(*jobs[0])
    r = None
    for _ in range(20000):
        r = srv.poll(t)
        if r is not None:
            break
        time.sleep(0.001)
    assert r is not None and r.status == 0
    with pytest.raises(abx.AbxError):
        srv.poll(t)  # the result was taken
    srv.close()
    with pytest.raises(abx.AbxError):
        abx.Server(ctx, 3, [])
