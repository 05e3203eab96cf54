"""Feature slicing (App. A): the library's exact integer-tick slice against
the oracle's set definition, hand-worked values, and the Libri-Light mode."""
import ctypes
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "slicing_handworked.txt")


def _lib():
    from paper_2505_02692_b300 import build
    lib = ctypes.CDLL(build.build())
    f = lib.abx_slice_frames
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    return f


def _product(f, t_on, t_off, dt, ll):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    rc = f(t_on, t_off, dt, int(ll), ctypes.byref(a), ctypes.byref(b))
    assert rc == 0
    return None if b.value < a.value else (a.value, b.value)


def _parse(tok):
    tok = tok.split()
    return None if tok == ["none"] else (int(tok[0]), int(tok[1]))


def test_golden_oracle_and_product():
    f = _lib()
    n = 0
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        times, plain, ll = line.split("|")
        t_on, t_off, dt = map(int, times.split())
        assert oracle.slice_frames(t_on, t_off, dt) == _parse(plain), line
        assert oracle.slice_frames(t_on, t_off, dt, True) == _parse(ll), line
        assert _product(f, t_on, t_off, dt, False) == _parse(plain), line
        assert _product(f, t_on, t_off, dt, True) == _parse(ll), line
        n += 1
    assert n == 5


def test_random_against_set_definition():
    f = _lib()
    rng = np.random.default_rng(0)
    for _ in range(3000):
        dt = int(rng.choice([10000, 20000, 40000, 80000, 12345]))
        t_on = int(rng.integers(0, 2_000_000))
        t_off = t_on + int(rng.integers(0, 400_000))
        if rng.random() < 0.3:   # snap to frame times and half steps
            t_on = (t_on // (dt // 2)) * (dt // 2) if dt % 2 == 0 else t_on
            t_off = max(t_on, (t_off // (dt // 2)) * (dt // 2) if dt % 2 == 0 else t_off)
        for ll in (False, True):
            assert _product(f, t_on, t_off, dt, ll) == oracle.slice_frames(t_on, t_off, dt, ll)


def test_bad_arguments():
    f = _lib()
    a, b = ctypes.c_int64(), ctypes.c_int64()
    assert f(10, 5, 20, 0, ctypes.byref(a), ctypes.byref(b)) == -1
    assert f(0, 5, 0, 0, ctypes.byref(a), ctypes.byref(b)) == -1
    with pytest.raises(ValueError):
        oracle.slice_frames(10, 5, 20)
