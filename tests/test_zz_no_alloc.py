"""The allocation-free entry point abx_dtw_pairs_noalloc.

It exists for callers that cannot allocate device memory (a pool they do not
own, a real-time loop, an allocator that already holds the device): the
library then works in one fixed static device array.  This file runs last so
that a failure here never hides the rest of the GPU suite.  The tests call
the entry point through the C ABI:

* twice in a row, with different pairs, comparing both results with the FP64
  oracle and with the allocating path (abx_distances, FP32 CUDA cores) within
  the FP32 parity tolerance; where FP32 and FP64 take optimal paths of
  different (near-tied) lengths the optimal costs must still agree;
* with a zero-norm frame: its pairs are NaN and the status call reports
  ABX_E_ZERO_NORM, and the next clean call clears the status;
* while its stream is being captured: rejected with ABX_E_UNSUPPORTED;
* with oversized requests: rejected before any GPU work."""
import numpy as np
import pytest

from paper_2505_02692_b300 import synth

from _common import TASKS, within_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_02692_b300 import abx as m
    m.lib()
    return m


def test_noalloc_matches_oracle_and_allocating_path_twice(abx):
    import torch
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
        d64, _, L64 = oracle.pair_distances(w.feats, w.offsets, sel[:, 0], sel[:, 1])
        ref_d, _, _, ref_len = dist.lookup(sel[:, 0], sel[:, 1])
        out = torch.full((len(sel),), float("nan"), device="cuda")
        ln = torch.zeros(len(sel), dtype=torch.int32, device="cuda")
        abx.abx_dtw_pairs_noalloc(feats, w.offsets, sel, out, ln)
        abx.abx_dtw_pairs_noalloc_check()
        got = out.cpu().numpy()
        got_len = ln.cpu().numpy().astype(np.int64)
        assert np.all(np.isfinite(got)), call
        # against the oracle: distance where the path length agrees, optimal
        # cost (distance x length) where FP32 picked a near-tied other length
        same = got_len == L64
        ok = np.where(same, within_tol(got, d64),
                      within_tol(got.astype(np.float64) * got_len, d64 * L64))
        assert ok.all(), (call, sel[~ok][:3], got[~ok][:3], d64[~ok][:3])
        assert np.mean(~same) <= 1e-3, (call, int(np.sum(~same)))
        # against the allocating entry point, the same way
        same_r = got_len == ref_len
        ok_r = np.where(same_r, within_tol(got, ref_d),
                        within_tol(got.astype(np.float64) * got_len,
                                   ref_d.astype(np.float64) * ref_len))
        assert ok_r.all(), call
        print(f"call {call}: {len(sel)} pairs, max |d - d64| {np.max(np.abs(got - d64)):.2e}, "
              f"{int(np.sum(~same))} with another optimal length than the oracle's")


def test_noalloc_zero_norm_frame_is_reported(abx):
    import torch

    rng = np.random.default_rng(5)
    offs = np.array([0, 3, 7, 12], dtype=np.int64)
    f = rng.standard_normal((12, 64)).astype(np.float32)
    f[4] = 0.0                                   # second frame of item 1
    feats = torch.from_numpy(f).cuda()
    pairs = np.array([[0, 1], [0, 2], [1, 2], [2, 0]], dtype=np.int64)
    out = torch.zeros(4, device="cuda")
    abx.abx_dtw_pairs_noalloc(feats, offs, pairs, out)
    with pytest.raises(abx.AbxError) as e:
        abx.abx_dtw_pairs_noalloc_check()
    assert e.value.code == -2                    # ABX_E_ZERO_NORM
    got = out.cpu().numpy()
    assert np.isnan(got[0]) and np.isnan(got[2])
    assert np.all(np.isfinite(got[[1, 3]]))
    # the next call starts from a clean status
    f[4] = 1.0
    abx.abx_dtw_pairs_noalloc(torch.from_numpy(f).cuda(), offs, pairs, out)
    abx.abx_dtw_pairs_noalloc_check()
    assert np.all(np.isfinite(out.cpu().numpy()))


def test_noalloc_refuses_stream_capture(abx):
    import torch

    offs = np.array([0, 4, 9], dtype=np.int64)
    feats = torch.randn(9, 32, device="cuda")
    pairs = np.array([[0, 1]], dtype=np.int64)
    out = torch.zeros(1, device="cuda")
    abx.abx_dtw_pairs_noalloc(feats, offs, pairs, out)   # device set-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    x = torch.zeros(1, device="cuda")
    err = None
    with torch.cuda.graph(g):
        x.add_(1.0)
        try:
            abx.abx_dtw_pairs_noalloc(feats, offs, pairs, out)
        except abx.AbxError as e:
            err = e
    assert err is not None and err.code == -5          # ABX_E_UNSUPPORTED
    abx.abx_dtw_pairs_noalloc(feats, offs, pairs, out)   # usable afterwards
    abx.abx_dtw_pairs_noalloc_check()
    assert np.isfinite(out.cpu().numpy()).all()


def test_noalloc_rejects_oversized_requests(abx):
    import torch

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
