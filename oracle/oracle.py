"""FP64 CPU oracle: distances, cells, cell scores and collapse.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Everything is the
plain definition from arXiv 2505.02692 written out, with library primitives
(sorting, dicts) as steps and no blocking or fusion:

* cells      -- Sec. 2 (definitions of on / by / across; Fig. 1 caption;
                Table 1): a triple (a, b, x) is valid when ``on`` is equal for
                a and x and different for b, every ``by`` attribute is equal
                for all three, and the ``across`` attribute is equal for a and
                b and different for x.  A cell gathers the triples of one
                (on_ax, on_b, by values[, across_ab, across_x]) combination.
* cell score -- Sec. 2, equation for D_C: mean over the cell's triples of
                1[d(a,x) < d(b,x)] + 1/2 1[d(a,x) = d(b,x)].  Kept as the exact
                integer numerator N = sum(2*win + tie) over the count |C|.
* collapse   -- Sec. 2 (average over contexts, then speakers, then phonemes;
                or a weighting by cell size) and Sec. 3.1 ``collapse(levels)``.
                Error = 1 - D.

Readings where the paper is silent (each also listed in the design notes):
  * a == x is not a triple (the same token cannot be both); within-style
    cells need at least two items of the on_ax value.
  * d(x, y) takes x as the DTW rows.
  * The unweighted collapse averages, level by level, over the listed
    attributes, summing in increasing order of the level's attribute codes
    (lexicographic in the order the level lists them; an across attribute
    contributes the ordered pair (across_ab, across_x)).  After the last
    level, the remaining entries are averaged in increasing order of
    (on_ax, on_b, remaining by attributes in ``by`` order, across pair).
  * The weighted collapse is sum(N) / sum(2|C|).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

MODE_DTW = 0
MODE_MEAN = 1
ANGULAR, COSINE, EUCLIDEAN, KL = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "abx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile abx_oracle.c into oracle/liboracle.so with gcc (FP64, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = [
            "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
            "-shared", "-fPIC", "-o", tmp, _SRC, "-lm",
        ]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        f32p = ctypes.POINTER(ctypes.c_float)
        f64p = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.abxo_angular.restype = ctypes.c_double
        lib.abxo_angular.argtypes = [f32p, f32p, ctypes.c_int64]
        lib.abxo_frame_dists.restype = None
        lib.abxo_frame_dists.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64,
                                         ctypes.c_int64, f64p]
        lib.abxo_dtw.restype = ctypes.c_int
        lib.abxo_dtw.argtypes = [f64p, ctypes.c_int64, ctypes.c_int64, f64p, i64p]
        lib.abxo_pair_distances.restype = ctypes.c_int
        lib.abxo_pair_distances.argtypes = [
            f32p, i64p, ctypes.c_int64, ctypes.c_int64, i64p, i64p, ctypes.c_int, ctypes.c_int,
            f64p, f64p, i64p, ctypes.c_int,
        ]
        lib.abxo_distance.restype = ctypes.c_double
        lib.abxo_distance.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_int]
        lib.abxo_max_threads.restype = ctypes.c_int
        lib.abxo_max_threads.argtypes = []
        _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def max_threads() -> int:
    """OpenMP threads the oracle uses for pair batches."""
    return int(_load().abxo_max_threads())


# ---------------------------------------------------------------- distances

def angular(u, v) -> float:
    """d(u, v) = arccos(cos angle(u, v)) / pi in FP64 (Sec. 3.1 "angular")."""
    u = np.ascontiguousarray(u, dtype=np.float32).ravel()
    v = np.ascontiguousarray(v, dtype=np.float32).ravel()
    assert u.shape == v.shape
    return float(_load().abxo_angular(_p(u, ctypes.c_float), _p(v, ctypes.c_float), u.size))


def distance(u, v, kind: int = ANGULAR) -> float:
    """Frame distance in FP64: ANGULAR, COSINE (1 - cos), EUCLIDEAN or KL (the
    symmetrised Kullback-Leibler divergence of the frames read as
    distributions: components must be positive, each frame is divided by its
    sum; NaN otherwise)."""
    u = np.ascontiguousarray(u, dtype=np.float32).ravel()
    v = np.ascontiguousarray(v, dtype=np.float32).ravel()
    assert u.shape == v.shape
    return float(_load().abxo_distance(_p(u, ctypes.c_float), _p(v, ctypes.c_float), u.size,
                                       int(kind)))


def frame_dists(X, Y) -> np.ndarray:
    """Matrix of angular distances, X frames on rows, Y frames on columns."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    out = np.empty((X.shape[0], Y.shape[0]), dtype=np.float64)
    _load().abxo_frame_dists(_p(X, ctypes.c_float), X.shape[0], _p(Y, ctypes.c_float),
                             Y.shape[0], X.shape[1], _p(out, ctypes.c_double))
    return out


def dtw(dmat) -> Tuple[float, int]:
    """DTW (Sec. 3.2) over a given distance matrix: (optimal cost, path length).

    Among equal-cost predecessors the shorter path wins."""
    d = np.ascontiguousarray(dmat, dtype=np.float64)
    cost = ctypes.c_double()
    ln = ctypes.c_int64()
    rc = _load().abxo_dtw(_p(d, ctypes.c_double), d.shape[0], d.shape[1],
                          ctypes.byref(cost), ctypes.byref(ln))
    if rc:
        raise ValueError("empty DTW input")
    return cost.value, int(ln.value)


def pair_distances(feats, offsets, px, py, mode: int = MODE_DTW, nthreads: int = 0,
                   kind: int = ANGULAR):
    """Distances of ordered item pairs (px[k] rows, py[k] columns).

    Returns (dist, cost, length) arrays; dist = cost / length for DTW and the
    angular distance of the mean frames for MEAN mode."""
    feats = np.ascontiguousarray(feats, dtype=np.float32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    px = np.ascontiguousarray(px, dtype=np.int64)
    py = np.ascontiguousarray(py, dtype=np.int64)
    n = px.size
    dist = np.empty(n, dtype=np.float64)
    cost = np.empty(n, dtype=np.float64)
    ln = np.empty(n, dtype=np.int64)
    if n:
        rc = _load().abxo_pair_distances(
            _p(feats, ctypes.c_float), _p(offsets, ctypes.c_int64), feats.shape[1], n,
            _p(px, ctypes.c_int64), _p(py, ctypes.c_int64), int(mode), int(kind),
            _p(dist, ctypes.c_double), _p(cost, ctypes.c_double), _p(ln, ctypes.c_int64),
            int(nthreads))
        if rc:
            raise ValueError("oracle pair distance failed (empty item?)")
    return dist, cost, ln


# -------------------------------------------------------------------- cells

@dataclass
class Cell:
    """One ABX cell: the triples (a, b, x) with a in A, b in B, x in X, a != x."""
    P: int                       # on value shared by a and x
    Q: int                       # on value of b
    by: Tuple[int, ...]          # by values (in the order of ``by``)
    across: Optional[Tuple[int, int]]  # (across_ab, across_x) or None
    A: List[int] = field(default_factory=list)
    B: List[int] = field(default_factory=list)
    X: List[int] = field(default_factory=list)

    @property
    def count(self) -> int:
        """|C|: number of triples, a == x excluded (sum over x of |A minus x| |B|;
        |X| (|A| - 1) |B| when X = A, |X| |A| |B| when they are disjoint)."""
        a = set(self.A)
        return sum(len(self.A) - (x in a) for x in self.X) * len(self.B)


def enumerate_cells(labels, on: int, by: Sequence[int] = (), across: Optional[int] = None
                    ) -> List[Cell]:
    """All non-empty cells of the task (Sec. 2 conditions, Sec. 3.1 ``Task``).

    ``labels`` is an (n_items, n_attr) integer array; ``on``, ``by`` and
    ``across`` are attribute (column) indices; at most one across attribute."""
    labels = np.asarray(labels)
    n = labels.shape[0]
    groups: Dict[Tuple[int, ...], List[int]] = {}
    for i in range(n):
        gkey = tuple(int(labels[i, b]) for b in by)
        groups.setdefault(gkey, []).append(i)
    cells: List[Cell] = []
    for gkey in sorted(groups):
        part: Dict[Tuple[int, int], List[int]] = {}
        for i in groups[gkey]:
            p = int(labels[i, on])
            s = int(labels[i, across]) if across is not None else 0
            part.setdefault((p, s), []).append(i)
        ons = sorted({p for (p, _) in part})
        sps = sorted({s for (_, s) in part})
        for P in ons:
            for Q in ons:
                if P == Q:
                    continue
                for s_ab in sps:
                    A = part.get((P, s_ab))
                    B = part.get((Q, s_ab))
                    if not A or not B:
                        continue
                    if across is None:
                        if len(A) < 2:
                            continue
                        cells.append(Cell(P, Q, gkey, None, list(A), list(B), list(A)))
                    else:
                        for s_x in sps:
                            if s_x == s_ab:
                                continue
                            X = part.get((P, s_x))
                            if not X:
                                continue
                            cells.append(Cell(P, Q, gkey, (s_ab, s_x), list(A), list(B),
                                              list(X)))
    return cells


def needed_pairs(cells: Iterable[Cell]) -> List[Tuple[int, int]]:
    """Ordered pairs (x, y) whose distance some triple compares."""
    need = set()
    for c in cells:
        for x in c.X:
            for a in c.A:
                if a != x:
                    need.add((x, a))
            for b in c.B:
                need.add((x, b))
    return sorted(need)


def score_cells(cells: Sequence[Cell], dist: Dict[Tuple[int, int], float]
                ) -> List[Tuple[int, int]]:
    """(N, |C|) per cell, N = sum over triples of 2*1[d(x,a)<d(x,b)] + 1[=]."""
    out = []
    for c in cells:
        num2 = 0
        cnt = 0
        for x in c.X:
            for a in c.A:
                if a == x:
                    continue
                dxa = dist[(x, a)]
                for b in c.B:
                    dxb = dist[(x, b)]
                    if dxa < dxb:
                        num2 += 2
                    elif dxa == dxb:
                        num2 += 1
                    cnt += 1
        assert cnt == c.count
        out.append((num2, cnt))
    return out


# ---------------------------------------------------------------- subsampling

M64 = (1 << 64) - 1
ROLE_A, ROLE_B, ROLE_X, ROLE_XACROSS = 0, 1, 2, 3


def splitmix64(x: int) -> int:
    """SplitMix64 output for state x (Steele, Lea & Flood, OOPSLA 2014; the
    generator of Java's SplittableRandom): add the golden-ratio increment,
    then two xor-shift-multiply rounds and a final xor-shift."""
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def fold(values) -> int:
    """Hash of a sequence of non-negative integers: h <- splitmix64(h xor v)."""
    h = 0
    for v in values:
        h = splitmix64(h ^ (int(v) & M64))
    return h


def subsample_cells(cells: Sequence[Cell], max_size_group: int = 0, max_x_across: int = 0,
                    seed: int = 0) -> List[Cell]:
    """The two subsampling methods of the Subsampler (Sec. 3.1, after
    Libri-Light), as a seeded, order-free draw.

    max_x_across (across tasks only): among the cells that share (by values,
    on_ax, on_b, across_ab), keep the max_x_across ones whose across_x value
    v has the smallest splitmix64(fold(seed, 3, by..., on_ax, on_b, across_ab)
    xor v), ties by v.
    max_size_group: in each remaining cell, each of A, B and X (roles 0, 1, 2)
    with more than max_size_group items keeps the max_size_group items i with
    the smallest splitmix64(fold(seed, role, by..., on_ax, on_b, across_ab,
    across_x) xor i), ties by i (across values 0, 0 for tasks without an
    across attribute).  Item numbers i are the items' rows in the labels.
    A cell left without a triple is dropped.  0 disables a method."""
    cells = list(cells)
    if max_x_across > 0:
        groups: Dict[tuple, List[Cell]] = {}
        for c in cells:
            if c.across is not None:
                groups.setdefault((c.by, c.P, c.Q, c.across[0]), []).append(c)
        keep = set()
        for (by, P, Q, s_ab), cs in groups.items():
            h = fold([seed, ROLE_XACROSS, *by, P, Q, s_ab])
            ranked = sorted(cs, key=lambda c: (splitmix64(h ^ c.across[1]), c.across[1]))
            keep.update(id(c) for c in ranked[:max_x_across])
        cells = [c for c in cells if c.across is None or id(c) in keep]
    out = []
    for c in cells:
        if max_size_group > 0:
            s_ab, s_x = c.across if c.across is not None else (0, 0)

            def pick(items, role):
                if len(items) <= max_size_group:
                    return list(items)
                h = fold([seed, role, *c.by, c.P, c.Q, s_ab, s_x])
                return sorted(items, key=lambda i: (splitmix64(h ^ i), i))[:max_size_group]

            c = Cell(c.P, c.Q, c.by, c.across, pick(c.A, ROLE_A), pick(c.B, ROLE_B),
                     pick(c.X, ROLE_X))
        if c.count > 0:
            out.append(c)
    return out


def collapse(cells: Sequence[Cell], scores: Sequence[Tuple[int, int]],
             levels: Sequence[Sequence[int]], by: Sequence[int] = (),
             across: Optional[int] = None, weighted: bool = False) -> float:
    """ABX error 1 - D from per-cell scores (Sec. 2 weighting; Sec. 3.1).

    ``levels`` lists, in order, the attribute groups averaged out one after
    the other (each a sequence of attribute indices from ``by`` / ``across``).
    """
    if weighted:
        num = sum(s[0] for s in scores)
        den = sum(2 * s[1] for s in scores)
        return 1.0 - num / den
    by = list(by)
    comps: List[Tuple[str, int]] = [("by", b) for b in by]
    if across is not None:
        comps.append(("across", across))

    def comp_of(attr: int) -> Tuple[str, int]:
        if attr in by:
            return ("by", attr)
        if across is not None and attr == across:
            return ("across", attr)
        raise ValueError(f"collapse level attribute {attr} is neither by nor across")

    # entry key: dict over remaining components plus on pair
    entries: List[Tuple[Dict, float]] = []
    for c, (num2, cnt) in zip(cells, scores):
        key = {("on", 0): c.P, ("on", 1): c.Q}
        for b, v in zip(by, c.by):
            key[("by", b)] = v
        if across is not None:
            key[("across", across)] = c.across
        entries.append((key, num2 / (2 * cnt)))

    remaining = list(comps)
    for level in levels:
        lcomps = [comp_of(a) for a in level]
        for lc in lcomps:
            if lc not in remaining:
                raise ValueError("attribute collapsed twice")
        keep = [("on", 0), ("on", 1)] + [c for c in remaining if c not in lcomps]
        groups: Dict[Tuple, List[Tuple[Tuple, float]]] = {}
        for key, val in entries:
            gk = tuple(key[c] for c in keep)
            order = tuple(key[c] for c in lcomps)
            groups.setdefault(gk, []).append((order, val))
        new_entries = []
        for gk, vals in groups.items():
            vals.sort(key=lambda t: t[0])
            s = 0.0
            for _, v in vals:
                s += v
            new_entries.append((dict(zip(keep, gk)), s / len(vals)))
        entries = new_entries
        remaining = [c for c in remaining if c not in lcomps]

    final_comps = [("on", 0), ("on", 1)] + remaining
    entries.sort(key=lambda e: tuple(e[0][c] for c in final_comps))
    s = 0.0
    for _, v in entries:
        s += v
    return 1.0 - s / len(entries)


def abx_error(feats, offsets, labels, on: int, by: Sequence[int] = (),
              across: Optional[int] = None, levels: Sequence[Sequence[int]] = (),
              mode: int = MODE_DTW, weighted: bool = False, nthreads: int = 0,
              kind: int = ANGULAR, max_size_group: int = 0, max_x_across: int = 0,
              seed: int = 0):
    """End to end: cells (optionally subsampled), needed distances, cell
    scores, collapsed error.

    Returns (error, cells, scores, dist_dict)."""
    cells = enumerate_cells(labels, on, by, across)
    if max_size_group > 0 or max_x_across > 0:
        cells = subsample_cells(cells, max_size_group, max_x_across, seed)
    pairs = needed_pairs(cells)
    px = np.array([p[0] for p in pairs], dtype=np.int64)
    py = np.array([p[1] for p in pairs], dtype=np.int64)
    dist, _, _ = pair_distances(feats, offsets, px, py, mode, nthreads, kind)
    dd = {p: float(v) for p, v in zip(pairs, dist)}
    scores = score_cells(cells, dd)
    err = collapse(cells, scores, levels, by, across, weighted) if cells else float("nan")
    return err, cells, scores, dd


# ------------------------------------------------------------------ slicing

def slice_frames(t_on: int, t_off: int, dt: int, libri_light: bool = False):
    """Frames kept for a unit spanning [t_on, t_off] (App. A, Eq. 1).

    Times are integers in one common unit (e.g. microseconds or samples).
    Follows the set definition directly: frame i has time t_i = dt/2 + i dt
    and is kept when t_on <= t_i <= t_off; scanned one frame at a time with
    doubled times so everything stays integral.  Returns (first, last),
    inclusive, or None when no frame is kept.  The Libri-Light convention
    drops the last kept frame (App. A, last paragraph)."""
    if dt <= 0 or t_on > t_off or t_on < 0:
        raise ValueError("need dt > 0 and 0 <= t_on <= t_off")
    kept = []
    i = 0
    while dt + 2 * dt * i <= 2 * t_off:
        if 2 * t_on <= dt + 2 * dt * i:
            kept.append(i)
        i += 1
    if libri_light and kept:
        kept = kept[:-1]
    if not kept:
        return None
    return kept[0], kept[-1]
