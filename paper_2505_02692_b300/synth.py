"""Seeded synthetic ABX workloads (features, item lengths, labels).

This module only draws inputs: it holds none of the method's arithmetic and
is shared by the tests, the oracle-side checks and the benchmark.

Generator (stands in for LibriSpeech dev-clean triphone features, which are
not available here): every item has a phone, a context and a speaker label,
drawn uniformly and independently; every frame of an item is

    mu[phone] + o[speaker] + eps,   mu ~ N(0, I), o ~ N(0, 0.3^2 I),
                                    eps ~ N(0, 0.5^2 I) i.i.d. per frame.

Item lengths follow either a uniform law on {lo..hi} or a law skewed toward
short items, P(T = k) proportional to exp(-(k - lo) / 6) on {lo..hi}.
Label columns: 0 = phone, 1 = context, 2 = speaker.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

PHONE, CONTEXT, SPEAKER = 0, 1, 2


@dataclass
class Workload:
    feats: np.ndarray      # (n_frames, dim) float32, items stored back to back
    offsets: np.ndarray    # (n_items + 1,) int64 CSR frame offsets
    labels: np.ndarray     # (n_items, 3) int32: phone, context, speaker
    seed: int
    name: str

    @property
    def n_items(self) -> int:
        return int(self.labels.shape[0])

    @property
    def dim(self) -> int:
        return int(self.feats.shape[1])

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)


def draw_lengths(rng: np.random.Generator, n: int, lo: int, hi: int, law: str) -> np.ndarray:
    ks = np.arange(lo, hi + 1)
    if law == "uniform":
        p = np.ones(ks.size)
    elif law == "skewed":
        p = np.exp(-(ks - lo) / 6.0)
    else:
        raise ValueError(law)
    p = p / p.sum()
    return rng.choice(ks, size=n, p=p).astype(np.int64)


def make_workload(n_items: int, dim: int, n_phone: int, n_context: int, n_speaker: int,
                  len_lo: int, len_hi: int, law: str = "uniform", seed: int = 0,
                  name: str = "custom", lengths: Optional[np.ndarray] = None,
                  noise: float = 0.5, spk_scale: float = 0.3) -> Workload:
    """Draw one synthetic workload (see the module docstring for the recipe;
    ``noise`` and ``spk_scale`` are the frame-noise and speaker-offset
    standard deviations, 0.5 and 0.3 in the standard recipe)."""
    rng = np.random.default_rng(seed)
    labels = np.stack([
        rng.integers(0, n_phone, n_items),
        rng.integers(0, n_context, n_items),
        rng.integers(0, n_speaker, n_items),
    ], axis=1).astype(np.int32)
    T = draw_lengths(rng, n_items, len_lo, len_hi, law) if lengths is None else \
        np.asarray(lengths, dtype=np.int64)
    offsets = np.zeros(n_items + 1, dtype=np.int64)
    np.cumsum(T, out=offsets[1:])
    n_frames = int(offsets[-1])
    mu = rng.standard_normal((n_phone, dim), dtype=np.float32)
    spk = (np.float32(spk_scale) * rng.standard_normal((n_speaker, dim), dtype=np.float32))
    frame_item = np.repeat(np.arange(n_items), T)
    feats = np.empty((n_frames, dim), dtype=np.float32)
    chunk = 1 << 16
    sd = np.float32(noise)
    for s in range(0, n_frames, chunk):
        e = min(n_frames, s + chunk)
        it = frame_item[s:e]
        buf = rng.standard_normal((e - s, dim), dtype=np.float32)
        buf *= sd
        buf += mu[labels[it, PHONE]]
        buf += spk[labels[it, SPEAKER]]
        feats[s:e] = buf
    return Workload(feats, offsets, labels, seed, name)


def tiny_within(seed: int = 0, noise: float = 0.5, spk_scale: float = 0.3) -> Workload:
    """400 items, 768-dim, lengths uniform 5-20, 10 phones x 20 contexts x 4 speakers."""
    return make_workload(400, 768, 10, 20, 4, 5, 20, "uniform", seed, "tiny-within-400x768",
                         noise=noise, spk_scale=spk_scale)


# Noise settings that make decisions hard (ABX error around 0.15 at dim 192),
# used by the parity tests so that wrong decisions cannot hide behind an
# error of exactly zero.  The standard recipe (0.5, 0.3) separates phones
# perfectly at these dimensions.
HARD = {"noise": 5.0, "spk_scale": 1.5}


def triphone_scale(seed: int = 0) -> Workload:
    """100k items, 768-dim, lengths 3-25 skewed short, 40 phones x 200 contexts x 40 speakers."""
    return make_workload(100_000, 768, 40, 200, 40, 3, 25, "skewed", seed,
                         "triphone-100k-768")


def medium(seed: int = 0, n_items: int = 3000, dim: int = 256, n_context: int = 6,
           n_speaker: int = 5, n_phone: int = 12, noise: float = 0.5,
           spk_scale: float = 0.3) -> Workload:
    """Mid-size case the oracle finishes in seconds yet spanning many tiles."""
    return make_workload(n_items, dim, n_phone, n_context, n_speaker, 3, 25, "skewed", seed,
                         f"medium-{n_items}x{dim}", noise=noise, spk_scale=spk_scale)


def gaussian_2d(n_per_class: int, shift: float, seed: int = 0) -> Workload:
    """Two 2-D Gaussian classes N(0, I) and N((s, s), I), one frame per item.

    Labels: phone = class, context = 0, speaker = 0 (Fig. 2 setting)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n_per_class, 2))
    b = rng.standard_normal((n_per_class, 2)) + shift
    feats = np.concatenate([a, b]).astype(np.float32)
    n = 2 * n_per_class
    labels = np.zeros((n, 3), dtype=np.int32)
    labels[n_per_class:, PHONE] = 1
    offsets = np.arange(n + 1, dtype=np.int64)
    return Workload(feats, offsets, labels, seed, f"gauss2d-shift{shift}")


# ------------------------------------------------- batched / served workloads

@dataclass
class TaskSpec:
    """One task of a batched or served workload (drawn by the functions below)."""
    n_items: int
    dim: int
    n_phone: int
    n_context: int
    n_speaker: int
    len_lo: int
    len_hi: int
    seed: int
    name: str


def batched_specs(seed: int = 0, n_tasks: int = 64, items=(1_000, 50_000),
                  dims=(256, 512, 768, 1024), lengths=(3, 40), phones=(10, 60),
                  n_context: int = 20, n_speaker: int = 4) -> list:
    """Ragged independent tasks: item counts log-uniform on `items`, dimension
    uniform over `dims`, lengths skewed short on `lengths`, phone count
    uniform on `phones`; context and speaker counts fixed."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_tasks):
        n = int(np.exp(rng.uniform(np.log(items[0]), np.log(items[1]))))
        dim = int(rng.choice(dims))
        nph = int(rng.integers(phones[0], phones[1] + 1))
        out.append(TaskSpec(n, dim, nph, n_context, n_speaker, lengths[0], lengths[1],
                            seed * 1000 + k, f"task{k}-{n}x{dim}"))
    return out


def make_task_device(spec: TaskSpec, device="cuda", noise: float = 0.5,
                     spk_scale: float = 0.3, feat_seed: Optional[int] = None):
    """Draw a task of the standard recipe with its frames on a CUDA device
    (torch, seeded): returns (feats tensor, offsets, labels) with offsets and
    labels as numpy arrays.  Lengths and labels come from numpy as in
    make_workload (seed spec.seed); frames from torch's generator on the
    device (seed feat_seed, default spec.seed), so several feature draws can
    share one item set, like the layers of one feature dump."""
    import torch
    rng = np.random.default_rng(spec.seed)
    labels = np.stack([
        rng.integers(0, spec.n_phone, spec.n_items),
        rng.integers(0, spec.n_context, spec.n_items),
        rng.integers(0, spec.n_speaker, spec.n_items),
    ], axis=1).astype(np.int32)
    T = draw_lengths(rng, spec.n_items, spec.len_lo, spec.len_hi, "skewed")
    offsets = np.zeros(spec.n_items + 1, dtype=np.int64)
    np.cumsum(T, out=offsets[1:])
    g = torch.Generator(device=device)
    g.manual_seed(spec.seed if feat_seed is None else feat_seed)
    mu = torch.randn(spec.n_phone, spec.dim, generator=g, device=device)
    spk = spk_scale * torch.randn(spec.n_speaker, spec.dim, generator=g, device=device)
    item = torch.repeat_interleave(torch.arange(spec.n_items, device=device),
                                   torch.as_tensor(T, device=device))
    lab = torch.as_tensor(labels, device=device, dtype=torch.int64)
    feats = noise * torch.randn(int(offsets[-1]), spec.dim, generator=g, device=device)
    feats += mu[lab[item, PHONE]]
    feats += spk[lab[item, SPEAKER]]
    return feats.contiguous(), offsets, labels


def served_dumps(seed: int = 0, n_dumps: int = 42, items=(2_000, 100_000),
                 dims=(512, 768, 1024, 1280), lengths=(3, 25), n_phone: int = 40,
                 n_context: int = 200, n_speaker: int = 40) -> list:
    """Feature dumps of a serving workload: item counts log-uniform on
    `items`, dimension uniform over `dims`, lengths skewed short; each dump's
    layers share its items (see make_task_device's feat_seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for d in range(n_dumps):
        n = int(np.exp(rng.uniform(np.log(items[0]), np.log(items[1]))))
        dim = int(rng.choice(dims))
        out.append(TaskSpec(n, dim, n_phone, n_context, n_speaker, lengths[0], lengths[1],
                            seed * 1000 + d, f"dump{d}-{n}x{dim}"))
    return out
