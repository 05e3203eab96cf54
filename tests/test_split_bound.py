"""The cosine error bound behind every distance interval, checked on the CPU.

The library's bound (abx_cosine_error_bound) states a model: the FP32 path
splits each frame, scaled by 2^14, into two FP16 halves v = hi + lo and forms
hi*hi and hi*lo + lo*hi on the tensor cores in two accumulators, dropping
lo*lo; each MMA instruction of K products adds them to the FP32 accumulator
with every addend aligned to the largest exponent and truncated, and the
result truncated (the
behaviour measured on earlier tensor cores by Fasi, Higham, Mikaitis and
Pranesh, PeerJ Comput. Sci. 2021).  Here that model is emulated exactly in
numpy on adversarial vectors -- every component just under half an FP16 unit
above an FP16 number, all of one sign, so that the lo halves are as large as
they get and every truncation errs the same way -- and the emulated cosine is
required to lie within the library's bound of the exact cosine of the stored
vectors.  A bound that left out a term (the dropped lo*lo, the three passes
of the split, the inverse-norm rounding) or a split with wider halves (BF16,
whose lo*lo term reaches 2^-16) fails here.
"""
import math

import numpy as np
import pytest
import torch

from paper_2505_02692_b300 import abx

FP32_SIMT, FP32, BF16, FP8 = 0, 1, 2, 3
HALF_MIN = 2.0 ** -14


def f16_split(v):
    """FP16 halves of float32 v (already scaled), halves below FP16's normal
    range stored as zero, as the pack kernel stores them."""
    v = np.asarray(v, dtype=np.float32)
    hi = v.astype(np.float16)
    hi[np.abs(hi.astype(np.float64)) < HALF_MIN] = 0
    r = (v - hi.astype(np.float32)).astype(np.float32)  # exact (Sterbenz)
    lo = r.astype(np.float16)
    lo[np.abs(lo.astype(np.float64)) < HALF_MIN] = 0
    return hi.astype(np.float64), lo.astype(np.float64)


def bf16(x):
    """Round float32 to bfloat16 (nearest, ties to even), returned as float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def e4m3(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(
        torch.float8_e4m3fn).to(torch.float64).numpy()


def trunc_f32(x):
    """Round a float64 toward zero to float32."""
    f = np.float32(x)
    if abs(float(f)) > abs(x):
        f = np.nextafter(f, np.float32(0.0))
    return float(f)


def mma_step(acc, prods):
    """One MMA instruction under the model: the accumulator and the exact
    products aligned to the largest exponent, each truncated toward zero to
    24 bits below it, added exactly, the sum truncated to float32."""
    ops = [acc] + [float(p) for p in prods]
    mx = max(abs(o) for o in ops)
    if mx == 0.0:
        return 0.0
    e = math.frexp(mx)[1]            # mx in [2^(e-1), 2^e)
    q = math.ldexp(1.0, e - 24)
    s = math.fsum(math.trunc(o / q) * q for o in ops)
    return trunc_f32(s)


def model_dot(pairs_of_vectors, k):
    """Dot product of operand streams through k-product MMA instructions; the
    streams are lists of (a, b) vectors accumulated in the kernel's order:
    per k step, every stream's k products in turn."""
    n = len(pairs_of_vectors[0][0])
    acc = 0.0
    for k0 in range(0, n, k):
        for a, b in pairs_of_vectors:
            acc = mma_step(acc, a[k0:k0 + k] * b[k0:k0 + k])
    return acc


def inv_norm_f32(q):
    """1/|q| the way the pack kernel forms it: sum of squares in float32
    (lane chains, then a tree), square root, division."""
    q32 = np.asarray(q, dtype=np.float32)
    lanes = np.zeros(32, dtype=np.float32)
    for c in range(len(q32)):
        lanes[c % 32] = np.float32(lanes[c % 32] + q32[c] * q32[c])
    while len(lanes) > 1:
        lanes = (lanes[: len(lanes) // 2] + lanes[len(lanes) // 2:]).astype(np.float32)
    return np.float32(1.0) / np.sqrt(lanes[0], dtype=np.float32)


def exact_cos(q1, q2):
    num = math.fsum(q1 * q2)         # products of float32 values are exact in float64
    return num / math.sqrt(math.fsum(q1 * q1) * math.fsum(q2 * q2))


def adversarial(rng, n, dim):
    """Positive vectors (scaled units, |v| ~ 2^14) whose components sit 0.49
    of an FP16 unit above an FP16 number: lo = +0.49 ulp everywhere."""
    out = []
    for _ in range(n):
        m = rng.uniform(300.0, 900.0, dim).astype(np.float16).astype(np.float64)
        ulp = np.spacing(m.astype(np.float16)).astype(np.float64)
        out.append((m + 0.49 * ulp).astype(np.float32))
    return out


@pytest.fixture(scope="module")
def bounds():
    return {p: abx.cosine_error_bound(p, 768) for p in (FP32_SIMT, FP32, BF16, FP8)}


def test_split_halves_and_dropped_term():
    rng = np.random.default_rng(1)
    vs = adversarial(rng, 6, 768)
    for v in vs:
        hi, lo = f16_split(v)
        assert np.all(lo > 0)                       # adversarial: lo of one sign
        assert np.all(np.abs(lo) <= 2.0 ** -11 * (1 + 2.0 ** -11) * np.abs(v))
        assert np.array_equal(hi + lo, v.astype(np.float64))  # 22 bits hold v exactly
    for v1, v2 in zip(vs[:-1], vs[1:]):
        _, l1 = f16_split(v1)
        _, l2 = f16_split(v2)
        rel = math.fsum(l1 * l2) / (np.linalg.norm(v1) * np.linalg.norm(v2))
        assert rel <= 2.0 ** -22 * (1 + 2.0 ** -9)
        assert rel > 0.2 * 2.0 ** -22               # and the case is near the worst


def test_bf16_split_would_exceed_the_fp32_bound(bounds):
    """A BF16 split (8-bit halves) drops lo*lo terms near 2^-16 on vectors
    built the same way for BF16: far above the split term the bound allows."""
    rng = np.random.default_rng(2)
    vs = []
    for _ in range(2):
        m = bf16(rng.uniform(0.5, 1.5, 768).astype(np.float32))
        ulp = np.ldexp(1.0, np.frexp(m)[1] - 8)       # BF16 unit in the last place
        vs.append((m + 0.49 * ulp).astype(np.float32))
    lows = [bf16((v - bf16(v)).astype(np.float32)) for v in vs]
    assert np.all(lows[0] > 0) and np.all(lows[1] > 0)
    rel = math.fsum(lows[0] * lows[1]) / (np.linalg.norm(vs[0]) * np.linalg.norm(vs[1]))
    assert rel > 2.0 ** -18                       # ~ (0.49 * 2^-7)^2 per unit norms
    assert rel > 16 * 2.0 ** -22 * (1 + 2.0 ** -9)


@pytest.mark.parametrize("prec", [FP32, BF16, FP8])
def test_model_cosine_within_bound(bounds, prec):
    rng = np.random.default_rng(10 + prec)
    vs = adversarial(rng, 4, 768)
    worst = 0.0
    for i in range(len(vs)):
        for j in range(i + 1, len(vs)):
            x, y = vs[i], vs[j]
            if prec == FP32:
                hx, lx = f16_split(x)
                hy, ly = f16_split(y)
                qx, qy = hx + lx, hy + ly
                # hi*hi and the cross terms in separate accumulators, added
                # once in float32 (round to nearest)
                acc = float(np.float32(model_dot([(hx, hy)], 16)) +
                            np.float32(model_dot([(hx, ly), (lx, hy)], 16)))
            elif prec == BF16:
                qx, qy = bf16(x), bf16(y)
                acc = model_dot([(qx, qy)], 16)
            else:
                sx = 448.0 / np.max(np.abs(x)) * np.linalg.norm(x)
                sy = 448.0 / np.max(np.abs(y)) * np.linalg.norm(y)
                qx = e4m3(x / np.linalg.norm(x) * sx)
                qy = e4m3(y / np.linalg.norm(y) * sy)
                acc = model_dot([(qx, qy)], 32)
            c = np.float32(np.float32(acc) * inv_norm_f32(qx)) * inv_norm_f32(qy)
            err = abs(float(c) - exact_cos(qx, qy))
            worst = max(worst, err)
            assert err <= bounds[prec], (prec, err, bounds[prec])
    if prec == FP32:
        # the hi*hi products lose their low bits to the aligned truncation,
        # all in one direction: a visible part of the bound
        assert worst > 0.02 * bounds[prec], (prec, worst, bounds[prec])


def test_bound_formula_terms(bounds):
    """The bound grows with the dimension and orders the precisions as the
    model does (three passes for the split, half the instructions for FP8)."""
    assert bounds[FP32] > bounds[BF16] > bounds[FP8] > 0
    assert bounds[FP32_SIMT] < bounds[BF16]
    assert abx.cosine_error_bound(FP32, 1536) > 1.9 * bounds[FP32]
    assert abx.cosine_error_bound(FP32, 700) == bounds[FP32]   # padded to 768
    with pytest.raises(abx.AbxError):
        abx.cosine_error_bound(7, 768)
