"""Host-side checks of the allocation-free entry point (no GPU needed): the
Python binding rejects buffers the C side cannot check, and the C side
rejects item offsets outside the feature matrix before any CUDA call."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2505_02692_b300 import abx


class FakeCuda:
    """Stands in for a CUDA tensor (attributes the binding's checks read)."""

    def __init__(self, shape, dtype, contiguous=True, device="cuda:0"):
        self.shape, self.dtype, self._c, self.device = tuple(shape), dtype, contiguous, device
        self.is_cuda = True

    def dim(self):
        return len(self.shape)

    def numel(self):
        return int(np.prod(self.shape))

    def is_contiguous(self):
        return self._c


def test_binding_rejects_bad_buffers():
    f32, i32 = torch.float32, torch.int32
    feats = FakeCuda((100, 8), f32)
    dist = FakeCuda((10,), f32)
    ok = dict(feats=feats, dist=dist, length=FakeCuda((10,), i32), n_pairs=10)
    abx._check_noalloc_buffers(**ok)                       # accepted
    bad = [
        dict(ok, feats=torch.zeros(100, 8)),               # host tensor
        dict(ok, feats=FakeCuda((100, 8), torch.float64)), # wrong dtype
        dict(ok, feats=FakeCuda((800,), f32)),             # not 2-D
        dict(ok, feats=FakeCuda((100, 8), f32, contiguous=False)),
        dict(ok, dist=FakeCuda((9,), f32)),                # too short
        dict(ok, dist=FakeCuda((10,), torch.float16)),
        dict(ok, dist=torch.zeros(10)),
        dict(ok, length=FakeCuda((9,), i32)),              # too short
        dict(ok, length=FakeCuda((10,), torch.int64)),
        dict(ok, dist=FakeCuda((10,), f32, device="cuda:1")),
    ]
    for b in bad:
        with pytest.raises(ValueError):
            abx._check_noalloc_buffers(**b)


def test_c_side_rejects_offsets_outside_the_features():
    L = abx.lib()
    fake_feats = ctypes.c_void_p(16)       # never dereferenced: rejected first
    out = ctypes.c_void_p(16)
    pairs = np.array([[0, 1]], dtype=np.int64)
    P = ctypes.POINTER(ctypes.c_int64)
    for offs in ([0, 100, 10], [0, 5, 3, 10], [0, 12, 10]):
        o = np.array(offs, dtype=np.int64)
        pr = pairs if len(offs) == 3 else np.array([[1, 2]], dtype=np.int64)
        rc = L.abx_dtw_pairs_noalloc(fake_feats, 10, 8, o.ctypes.data_as(P), len(offs) - 1,
                                     pr.ctypes.data_as(P), 1, out, None, None)
        assert rc == -1, offs
        assert b"frame" in L.abx_last_error()
