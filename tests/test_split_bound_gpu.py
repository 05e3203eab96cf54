"""The cosine error bound on the tensor cores, with adversarial frames.

Every frame here has positive components only, so the FP32 accumulation's
roundings (truncations, if the hardware truncates) all err the same way, and
the frames are built so that the stored vector the kernels use is known:

* FP8: components are E4M3 values, the largest 448, so the pack's per-item
  scale maps them onto themselves and the stored vector is the frame;
* BF16: components are BF16 values and the frame has unit norm to within
  1e-4, so normalising moves no component off its BF16 value;
* FP32 split: components sit 0.49 of an FP16 unit above an FP16 number at
  the 2^14 scale of the split, so every lo half is as large as it gets and of
  one sign; the stored vector is then within 2^-22 of the frame.

For one-frame items the cosine distance 1 - c gives the kernel's cosine c,
which must lie within abx_cosine_error_bound of the exact cosine (for the
split, plus the stored vectors' angle to the frames, at most 1e-6 each).
Multi-frame items with the angular distance must have the FP64 oracle value
inside every interval [lo, hi], the FP32 split within the per-pair
tolerance, and with the recheck the oracle's ABX error."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2505_02692_b300 import synth

from _common import TASKS, oracle_run, within_tol

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


def _bf16(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def frames(kind, n, dim, rng):
    out = np.empty((n, dim), dtype=np.float32)
    for i in range(n):
        if kind == "fp8":
            v = torch.from_numpy(rng.uniform(20.0, 400.0, dim).astype(np.float32)).to(
                torch.float8_e4m3fn).to(torch.float32).numpy()
            v[rng.integers(dim)] = 448.0
        elif kind == "bf16":
            v = _bf16(rng.uniform(0.02, 0.05, dim) / 1.0)
            v = _bf16(v / np.sqrt(np.sum(v.astype(np.float64) ** 2)))
            for _ in range(4):       # adjust the largest component toward unit norm
                k = int(np.argmax(v))
                rest = np.sum(v.astype(np.float64) ** 2) - float(v[k]) ** 2
                v[k] = _bf16(np.sqrt(max(1.0 - rest, 0.0)))
            # |x| = 1 to 1e-4: normalising scales each component by at most
            # 5e-5, far inside half a BF16 unit (2^-9 relative)
            assert abs(np.sum(v.astype(np.float64) ** 2) - 1.0) < 1e-4
        else:
            # sum of squares below 2^28 before the last component (mean
            # square about 3.0e5 here), which then makes |v| = 2^14 exactly
            # enough that the pack's x / |x| * 2^14 gives v back
            m = rng.uniform(250.0, 800.0, dim).astype(np.float16)
            ulp = np.spacing(m).astype(np.float64)
            v = (m.astype(np.float64) + 0.49 * ulp)
            v[-1] = 0.0
            rest = 2.0 ** 28 - np.sum(v ** 2)
            assert rest > 0
            v[-1] = np.sqrt(rest)
            v = v.astype(np.float32)
        out[i] = v
    return out


def _one_frame_task(feats):
    n = feats.shape[0]
    labels = np.zeros((n, 3), dtype=np.int32)
    labels[n // 2:, synth.PHONE] = 1            # two phones, every pair needed
    offsets = np.arange(n + 1, dtype=np.int64)
    return synth.Workload(feats, offsets, labels, 0, "adversarial-1frame")


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_cosine_error_within_bound(abx, ctx, prec):
    rng = np.random.default_rng(7)
    dim = 768
    w = _one_frame_task(frames(prec, 24, dim, rng))
    on, by, across, _ = TASKS["within"]
    items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
    cells = abx.abx_build_cells(ctx, items, on, by, across)
    dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.PRECISIONS[prec],
                             distance=abx.COSINE)
    n = w.n_items
    px, py = np.triu_indices(n, 1)
    d, _, _, ln = dist.lookup(px, py)
    assert np.all(ln == 1)
    x = w.feats.astype(np.float64)
    c_exact = np.array([math.fsum(x[i] * x[j]) / math.sqrt(math.fsum(x[i] * x[i]) *
                                                             math.fsum(x[j] * x[j]))
                        for i, j in zip(px, py)])
    c_gpu = 1.0 - d.astype(np.float64)
    err = np.abs(c_gpu - c_exact)
    bound = abx.cosine_error_bound(abx.PRECISIONS[prec], dim)
    slack = 2e-6 if prec == "fp32" else 0.0      # angle of the split's stored vectors
    slack += 2.0 ** -24                          # rounding of d = 1 - c
    print(f"{prec}: max |c - c64| {err.max():.3e}, bound {bound:.3e} "
          f"({err.max() / bound:.3f} of it), cos in [{c_exact.min():.3f}, {c_exact.max():.3f}]")
    assert np.all(err <= bound + slack), (err.max(), bound)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_adversarial_intervals_hold_the_oracle(abx, ctx, prec):
    rng = np.random.default_rng(8)
    n, dim = 60, 768
    lengths = rng.integers(1, 7, n)
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    feats = frames("fp32" if prec == "fp32" else prec, int(offsets[-1]), dim, rng)
    # spread the cosines: scale a random half of each frame's components down
    mask = rng.random(feats.shape) < 0.5
    if prec == "fp8":
        feats = np.where(mask & (feats < 448.0), np.float32(16.0), feats)
    elif prec == "bf16":
        feats = np.where(mask, _bf16(feats * 0.25), feats).astype(np.float32)
    else:
        feats = np.where(mask, feats * np.float32(0.25), feats).astype(np.float32)
    labels = np.stack([rng.integers(0, 3, n), np.zeros(n), rng.integers(0, 2, n)],
                      1).astype(np.int32)
    w = synth.Workload(feats, offsets, labels, 8, "adversarial")
    for task in ("within", "across"):
        err_o, cells_o, scores_o, dd = oracle_run(w, task)
        on, by, across, levels = TASKS[task]
        items = abx.abx_load_items(ctx, w.feats, w.offsets, w.labels)
        cells = abx.abx_build_cells(ctx, items, on, by, across)
        dist = abx.abx_distances(ctx, items, cells, abx.DTW, abx.PRECISIONS[prec])
        pairs = np.array(sorted(dd), dtype=np.int64)
        want = np.array([dd[tuple(p)] for p in pairs])
        d, lo, hi, ln = dist.lookup(pairs[:, 0], pairs[:, 1])
        assert np.all(ln > 0)
        inside = (lo <= want) & (want <= hi)
        assert inside.all(), (prec, task, pairs[~inside][:3], lo[~inside][:3],
                              want[~inside][:3], hi[~inside][:3])
        if prec == "fp32":
            ok = within_tol(d, want)
            assert ok.all(), (pairs[~ok][:3], d[~ok][:3], want[~ok][:3])
        err, st = abx.abx_score(ctx, dist, cells, levels, recheck=True)
        assert err == err_o or (np.isnan(err) and np.isnan(err_o))
        print(f"{prec} {task}: max |d - d64| {np.max(np.abs(d - want)):.2e}, "
              f"mean interval width {np.mean(hi - lo):.2e}, "
              f"recheck pairs {st.n_recheck_pairs}")
