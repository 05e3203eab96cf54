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

# FP32 per-pair tolerance: 1e-5 relative, or the effect of a cosine error
# of COS_TOL through arccos, whichever is larger.  d = arccos(c) / pi has
# slope 1 / (pi sin(pi d)), so near-parallel frames (small d) amplify the
# cosine's FP32 rounding: FP32 dot products over a few hundred terms carry
# errors of order sqrt(dim) * 2^-24 ~ 1e-6, and at d = 0.04 that alone is
# 2.5e-5 of d.  Near d = 0 the bound is arccos(1 - COS_TOL) / pi.
REL_TOL = 1e-5
COS_TOL = 1e-6


def within_tol(got, want, rel=REL_TOL, cos_tol=COS_TOL):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    s = np.sin(np.pi * np.clip(want, 0.0, 1.0))
    cond = np.minimum(cos_tol / (np.pi * np.maximum(s, 1e-300)),
                      np.sqrt(2.0 * cos_tol) / np.pi)
    return np.abs(got - want) <= np.maximum(rel * np.abs(want), cond)


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
