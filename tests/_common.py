"""Helpers shared by the parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded synthetic inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2505_02692_b300 import synth

PHONE, CONTEXT, SPEAKER = synth.PHONE, synth.CONTEXT, synth.SPEAKER

# task name -> (on, by, across, collapse levels)
TASKS = {
    "within": (PHONE, (CONTEXT, SPEAKER), None, [(CONTEXT,), (SPEAKER,)]),
    "across": (PHONE, (CONTEXT,), SPEAKER, [(CONTEXT,), (SPEAKER,)]),
}

# FP32 per-pair tolerance: 1e-5 relative, with an absolute floor of 1e-6
# where the distance is below 1e-3 (arccos is ill-conditioned near cos = 1,
# where a 1-ulp FP32 cosine error alone moves d by ~1e-4 * sqrt(ulp)).
REL_TOL = 1e-5
ABS_FLOOR = 1e-6


def within_tol(got, want, rel=REL_TOL, floor=ABS_FLOOR):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    return np.abs(got - want) <= np.maximum(rel * np.abs(want), floor)


def oracle_run(w: synth.Workload, task: str, mode=oracle.MODE_DTW, weighted=False):
    on, by, across, levels = TASKS[task]
    err, cells, scores, dd = oracle.abx_error(w.feats, w.offsets, w.labels, on, by, across,
                                              levels, mode, weighted)
    return err, cells, scores, dd


def cell_table_oracle(cells, scores, n_by):
    """{(P, Q, s_ab, s_x, by...): (N, |C|)} from oracle cells."""
    out = {}
    for c, (num2, cnt) in zip(cells, scores):
        s_ab, s_x = c.across if c.across is not None else (0, 0)
        out[(c.P, c.Q, s_ab, s_x) + tuple(c.by)] = (num2, cnt)
    return out


def cell_table_product(keys, num2, cnt):
    return {tuple(int(v) for v in k): (int(a), int(b)) for k, a, b in zip(keys, num2, cnt)}
