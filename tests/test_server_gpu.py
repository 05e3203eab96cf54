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


# ------------------------------------------------------- failure handling
# Failures are made on the host (a malformed job, a zero-norm frame that the
# pack kernel reports as a status word, a cancellation, an injected
# allocation failure); none of them faults or stalls the GPU.  In each case
# every other job's result must equal the job run alone.

def _check_alone(abx, ctx_alone, jobs, res, skip=()):
    for k, r in enumerate(res):
        if k in skip:
            continue
        assert r.status == 0, (k, r.status)
        ref = _alone(abx, ctx_alone, jobs[k], abx.BF16)
        for q in range(2):
            e, t = ref[q]
            assert r.errors[q] == e or (np.isnan(r.errors[q]) and np.isnan(e)), (k, q)
            assert r.triplets[q] == t


def test_server_malformed_jobs_leave_the_others_unchanged(abx):
    jobs = _jobs(seed=5, n_dumps=2, layers=2)
    ctx_alone, ctx = abx.Context(0), abx.Context(0)
    srv = abx.Server(ctx, 3, _specs(abx), abx.DTW, abx.BF16, recheck=True, max_batch_jobs=8)
    feats, offs, labels = jobs[0]
    bad_offs = offs.copy()
    bad_offs[3] = bad_offs[2]                       # an item without frames
    bad_labels = labels.copy()
    bad_labels[5, 1] = -1                           # a negative label code
    tickets = [srv.submit(*jobs[0]), srv.submit(*jobs[1])]
    for f, o, lab in ((feats, bad_offs, labels), (feats, offs, bad_labels)):
        with pytest.raises(abx.AbxError) as e:
            srv.submit(f, o, lab)
        assert e.value.code == -1                   # refused, never queued
    # a zero-norm frame passes the host checks and is found on the GPU: the
    # shared batch it lands in fails, is split, and only this job fails
    zero = feats.copy()
    zero[int(offs[4])] = 0.0
    tickets.append(srv.submit(zero, offs, labels))
    tickets += [srv.submit(*j) for j in jobs[2:]]
    res = [srv.wait(t) for t in tickets]
    st = srv.stats
    srv.close()
    assert res[2].status == -2                      # ABX_E_ZERO_NORM
    assert st.failed == 1 and st.completed == len(tickets) - 1
    ordered = [jobs[0], jobs[1], None] + jobs[2:]
    _check_alone(abx, ctx_alone, ordered, res, skip=(2,))
    print(f"batches {st.batches}, split {st.retried}")


def test_server_cancel_a_queued_job(abx):
    jobs = _jobs(seed=6, n_dumps=2, layers=3)
    ctx_alone, ctx = abx.Context(0), abx.Context(0)
    # one executor and batches of one job: the later jobs wait in the queue
    srv = abx.Server(ctx, 3, _specs(abx), abx.DTW, abx.BF16, recheck=True, max_batch_jobs=1)
    tickets = [srv.submit(*j) for j in jobs]
    cancelled = None
    for k in range(len(tickets) - 1, 0, -1):
        try:
            srv.cancel(tickets[k])
            cancelled = k
            break
        except abx.AbxError as e:
            assert e.value.code == -6               # already admitted: not cancellable
    assert cancelled is not None
    res = [srv.wait(t) for t in tickets]
    st = srv.stats
    with pytest.raises(abx.AbxError):
        srv.cancel(tickets[0])                      # done (and taken): unknown ticket
    srv.close()
    assert res[cancelled].status == -7              # ABX_E_CANCELLED
    assert st.cancelled == 1 and st.completed == len(jobs) - 1
    _check_alone(abx, ctx_alone, jobs, res, skip=(cancelled,))


def test_server_injected_allocation_failure(abx):
    """The second batch creation fails as an allocation failure would.  The
    first job is taken into the first batch before the rest are submitted
    (otherwise all seven fit one batch and nothing is injected), and keeps
    the executor busy while they are queued, so the second batch usually
    holds several jobs: it is split and they run alone."""
    jobs = _jobs(seed=7, n_dumps=2, layers=3)
    ctx_alone, ctx = abx.Context(0), abx.Context(0)
    srv = abx.Server(ctx, 3, _specs(abx), abx.DTW, abx.BF16, recheck=True, max_batch_jobs=8,
                     fail_inject=2)
    big = synth.make_workload(6000, 512, 8, 4, 3, 3, 25, "skewed", seed=99, name="big",
                              **synth.HARD)
    t0 = srv.submit(big.feats, big.offsets, big.labels)
    t_end = time.monotonic() + 30.0
    while srv.stats.batches < 1 and time.monotonic() < t_end:
        time.sleep(0.0005)
    assert srv.stats.batches >= 1
    tickets = [srv.submit(*j) for j in jobs]
    res = [srv.wait(t) for t in tickets]
    assert srv.wait(t0).status == 0
    st = srv.stats
    srv.close()
    failed = [k for k, r in enumerate(res) if r.status != 0]
    if st.retried:
        assert not failed                           # split and run alone: all succeed
    else:                                           # the failed batch held one job
        assert len(failed) == 1 and res[failed[0]].status == -3
    _check_alone(abx, ctx_alone, jobs, res, skip=tuple(failed))
    print(f"batches {st.batches}, split {st.retried}, failed {failed}")


def test_server_batches_under_load(abx):
    """Jobs arriving while the executor is busy join one batch (just-in-time
    planning): more than one job per batch on average."""
    jobs = _jobs(seed=8, n_dumps=2, layers=4)
    ctx = abx.Context(0)
    srv = abx.Server(ctx, 3, _specs(abx), abx.DTW, abx.BF16, recheck=True, max_batch_jobs=8)
    big = synth.make_workload(6000, 512, 8, 4, 3, 3, 25, "skewed", seed=98, name="big",
                              **synth.HARD)
    t0 = srv.submit(big.feats, big.offsets, big.labels)
    tickets = [srv.submit(*j) for j in jobs]
    res = [srv.wait(t) for t in tickets]
    srv.wait(t0)
    st = srv.stats
    srv.close()
    assert all(r.status == 0 for r in res)
    assert st.batches < len(jobs) + 1
    assert max(r.batch_jobs for r in res) > 1
