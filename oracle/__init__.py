"""Plain, slow, FP64 CPU oracle for the fastabx distance/score path.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call
or execute anything in this package.  The product library under
``paper_2505_02692_b300`` never imports it and shares no code with it.

Contents (arXiv 2505.02692):
  * ``abx_oracle.c`` -- FP64 angular frame distance (Sec. 3.1), DTW dynamic
    programme (Sec. 3.2) normalised by the optimal path length, mean-pooled
    item distance (Sec. 3.2), batched over item pairs with OpenMP.
  * ``oracle.py`` -- feature slicing by onset/offset (App. A), the subsampler
    (Sec. 3.1, a seeded SplitMix64 draw), cell enumeration from the on/by/across conditions
    (Sec. 2, Fig. 1 caption, Table 1), the cell score D_C (Sec. 2 equation),
    and the collapse (Sec. 2 weighting paragraph; Sec. 3.1 ``collapse``).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(hand-worked values, brute force on tiny inputs, closed forms, invariants).
"""
from .oracle import (  # noqa: F401
    MODE_DTW,
    MODE_MEAN,
    ANGULAR,
    COSINE,
    EUCLIDEAN,
    KL,
    distance,
    Cell,
    angular,
    build,
    collapse,
    dtw,
    enumerate_cells,
    frame_dists,
    abx_error,
    max_threads,
    needed_pairs,
    pair_distances,
    score_cells,
    slice_frames,
    splitmix64,
    fold,
    subsample_cells,
)
