"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol include/abx.h declares, and fails cleanly (no fallback) without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(abx_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libabx():
    from paper_2505_02692_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libabx):
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(libabx, n), n


def test_version_and_error_string(libabx):
    libabx.abx_version.restype = ctypes.c_char_p
    libabx.abx_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in libabx.abx_version()
    assert isinstance(libabx.abx_last_error(), bytes)


def test_null_arguments_are_rejected(libabx):
    # argument checks run before any CUDA call
    assert libabx.abx_ctx_create(0, None) == -1
    assert libabx.abx_cells_get_info(None, None) == -1
    assert libabx.abx_dist_get_info(None, None) == -1
    assert libabx.abx_items_free(None) == 0
    assert libabx.abx_cells_free(None) == 0
    assert libabx.abx_dist_free(None) == 0


def test_binding_has_no_cpu_fallback():
    import torch
    from paper_2505_02692_b300 import abx
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(abx.AbxError):
        abx.Context(0)


def test_binding_names_match_abi():
    from paper_2505_02692_b300 import abx
    for n in ("abx_load_items", "abx_build_cells", "abx_distances", "abx_score",
              "abx_score_cells"):
        assert callable(getattr(abx, n))
