"""The allocation-free entry point abx_dtw_pairs_noalloc.

It exists for callers that cannot allocate device memory (a pool they do not
own, a real-time loop, an allocator that already holds the device): the
library then works in one fixed static device array.  This file runs last so
that a failure here never hides the rest of the GPU suite.  The test calls
the entry point through the C ABI twice in a row, with different pairs, and
compares both results with the allocating path (abx_distances, FP32 CUDA
cores) within the FP32 parity tolerance; oversized requests must be
rejected before any GPU work."""
import numpy as np
import pytest

from paper_2505_02692_b300 import synth

from _common import TASKS, within_tol

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_path_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_02692_b300 import abx
    import oracle

    w = synth.medium(seed=21, n_items=900, dim=192, n_context=3, n_speaker=3, n_phone=8,
                     **synth.HARD)
    ctx = abx.Context(0)
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    on, by, across, _ = TASKS["across"]
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.FP32_SIMT)
    needed = np.array(oracle.needed_pairs(oracle.enumerate_cells(w.labels, on, by, across)),
                      dtype=np.int64)
    rng = np.random.default_rng(3)
    feats = torch.from_numpy(w.feats).cuda()
    for call in range(2):
        sel = needed[rng.choice(len(needed), 4000, replace=False)]
        ref_d, _, _, ref_len = dist.lookup(sel[:, 0], sel[:, 1])
        out = torch.full((len(sel),), float("nan"), device="cuda")
        ln = torch.zeros(len(sel), dtype=torch.int32, device="cuda")
        abx.abx_dtw_pairs_noalloc(feats, w.offsets, sel, out, ln)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        got_len = ln.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        same_path = got_len == ref_len
        assert np.mean(same_path) > 0.999, call
        assert within_tol(got[same_path], ref_d[same_path]).all(), call


def test_noalloc_rejects_oversized_requests():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_02692_b300 import abx

    offs = np.array([0, 128, 256], dtype=np.int64)
    feats = torch.ones((256, 8), device="cuda")
    out = torch.empty(70000, device="cuda")
    with pytest.raises(abx.AbxError) as e:
        abx.abx_dtw_pairs_noalloc(feats, offs, np.zeros((70000, 2), np.int64), out)
    assert e.value.code == -5
    # 300 pairs of 128 x 128 frames exceed the 2^22 frame-pair scratch
    with pytest.raises(abx.AbxError) as e:
        abx.abx_dtw_pairs_noalloc(feats, offs, np.tile([[0, 1]], (300, 1)), out)
    assert e.value.code == -5
