"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each check is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand, a wrong tie rule or
normalisation, a wrong collapse order) fails at least one of them:

* hand-worked angular distances and DTW results (tests/golden/);
* the angular distance against an independent half-angle formula;
* DTW against brute force over every monotone path on tiny inputs;
* closed forms (single frames, one-row DTW, constant distance matrices);
* invariants (self-distance 0, symmetry, ranges, scale invariance, path
  length bounds, mean mode = DTW mode on single frames);
* cell enumeration against brute-force triple enumeration from the labels;
* the cell score (ties = 1/2, A/B swap = 1 - D without ties) and the
  collapse against a hand-worked example;
* the 2-D Gaussian experiment of Fig. 2 at zero shift (error 1/2) and a
  well-separated case (error 0).
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2505_02692_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frames(txt):
    return np.array([[float(v) for v in f.split()] for f in txt.split(";")], dtype=np.float32)


# ------------------------------------------------------------ golden values

def test_angular_golden():
    n = 0
    with open(os.path.join(GOLDEN, "angular_handworked.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            u, v, want = line.split(";")
            got = oracle.angular(_frames(u)[0], _frames(v)[0])
            # 1e-8: see the arccos conditioning note in test_dtw_golden
            assert abs(got - float(want)) < 1e-8, (line, got)
            n += 1
    assert n >= 5


def test_dtw_golden():
    n = 0
    with open(os.path.join(GOLDEN, "dtw_handworked.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            xs, ys, cost, ln, dist = line.split("|")
            X, Y = _frames(xs), _frames(ys)
            c, L = oracle.dtw(oracle.frame_dists(X, Y))
            # arccos is ill-conditioned at cos = 1: a last-bit error of the
            # FP64 cosine of parallel frames gives sqrt(2 * 2^-52) / pi ~ 7e-9
            assert abs(c - float(cost)) < 1e-8, line
            assert L == int(ln), line
            offs = np.array([0, len(X), len(X) + len(Y)], dtype=np.int64)
            d, c2, L2 = oracle.pair_distances(np.concatenate([X, Y]), offs, [0], [1])
            assert abs(d[0] - float(dist)) < 1e-8 and L2[0] == int(ln)
            n += 1
    assert n >= 6


def test_dtw_tie_rule_prefers_shorter_path():
    # golden line (b) again, explicitly: an up-first rule would give 1/6
    X = _frames("1 0 ; 0 1")
    Y = _frames("0 1 ; 0 1")
    c, L = oracle.dtw(oracle.frame_dists(X, Y))
    assert (c, L) == (0.5, 2)


# ------------------------------------------- independent angular formula

def test_angular_half_angle_formula():
    rng = np.random.default_rng(1)
    for dim in (2, 3, 17, 768):
        for _ in range(20):
            u = rng.standard_normal(dim).astype(np.float32)
            v = rng.standard_normal(dim).astype(np.float32)
            uu = u.astype(np.float64) / np.linalg.norm(u.astype(np.float64))
            vv = v.astype(np.float64) / np.linalg.norm(v.astype(np.float64))
            # theta = 2 atan2(|u^ - v^|, |u^ + v^|): a different computation
            theta = 2.0 * math.atan2(np.linalg.norm(uu - vv), np.linalg.norm(uu + vv))
            assert abs(oracle.angular(u, v) - theta / math.pi) < 1e-12


# ------------------------------------------------------------- brute force

def _paths(tx, ty):
    """Every monotone path from (0,0) to (tx-1,ty-1) with steps (1,0),(0,1),(1,1)."""
    out = []

    def rec(i, j, acc):
        acc = acc + [(i, j)]
        if i == tx - 1 and j == ty - 1:
            out.append(acc)
            return
        if i + 1 < tx:
            rec(i + 1, j, acc)
        if j + 1 < ty:
            rec(i, j + 1, acc)
        if i + 1 < tx and j + 1 < ty:
            rec(i + 1, j + 1, acc)

    rec(0, 0, [])
    return out


def test_dtw_brute_force_all_paths():
    rng = np.random.default_rng(2)
    checked = 0
    for tx in range(1, 6):
        for ty in range(1, 6):
            paths = _paths(tx, ty)
            for trial in range(6):
                if trial % 2:
                    d = rng.random((tx, ty))
                else:  # multiples of 1/8 produce many exact cost ties
                    d = rng.integers(0, 4, (tx, ty)) / 8.0
                best = None
                for p in paths:
                    s = 0.0
                    for (i, j) in p:   # same addition order as the recurrence
                        s = d[i, j] + s
                    key = (s, len(p))
                    if best is None or key < best:
                        best = key
                c, L = oracle.dtw(d)
                assert (c, L) == best, (tx, ty, d)
                checked += 1
    assert checked == 150


# --------------------------------------------------------------- closed forms

def test_dtw_single_frames_is_angular():
    rng = np.random.default_rng(3)
    for _ in range(10):
        u = rng.standard_normal((1, 64)).astype(np.float32)
        v = rng.standard_normal((1, 64)).astype(np.float32)
        offs = np.array([0, 1, 2], dtype=np.int64)
        d, c, L = oracle.pair_distances(np.concatenate([u, v]), offs, [0], [1])
        assert L[0] == 1 and d[0] == oracle.angular(u[0], v[0])


def test_dtw_one_row_is_row_mean():
    rng = np.random.default_rng(4)
    for n in range(1, 9):
        u = rng.standard_normal((1, 32)).astype(np.float32)
        Y = rng.standard_normal((n, 32)).astype(np.float32)
        dm = oracle.frame_dists(u, Y)
        c, L = oracle.dtw(dm)
        assert L == n and abs(c / L - dm.mean()) < 1e-14
        c2, L2 = oracle.dtw(dm.T.copy())
        assert (c2, L2) == (c, L)


def test_dtw_constant_matrix():
    for tx, ty in [(1, 1), (3, 5), (7, 2), (4, 4)]:
        d = np.full((tx, ty), 0.375)
        c, L = oracle.dtw(d)
        assert L == max(tx, ty) and c / L == 0.375


# ----------------------------------------------------------------- invariants

def test_invariants_random_items():
    rng = np.random.default_rng(5)
    dim = 48
    T = rng.integers(1, 12, 12)
    offs = np.concatenate([[0], np.cumsum(T)]).astype(np.int64)
    feats = rng.standard_normal((int(offs[-1]), dim)).astype(np.float32)
    n = len(T)
    px, py = zip(*[(i, j) for i in range(n) for j in range(n)])
    d, c, L = oracle.pair_distances(feats, offs, px, py)
    D = d.reshape(n, n)
    Lm = L.reshape(n, n)
    assert np.all(D >= 0) and np.all(D <= 1)
    assert np.all(np.abs(np.diag(D)) <= 1e-7)          # DTW(x, x) = 0
    assert np.array_equal(D, D.T)                       # symmetric
    assert np.array_equal(Lm, Lm.T)
    for i in range(n):
        for j in range(n):
            assert max(T[i], T[j]) <= Lm[i, j] <= T[i] + T[j] - 1
    # positive rescaling of any frame changes nothing; powers of two keep the
    # FP32 inputs exact, so the FP64 results must agree bit for bit
    scale = np.exp2(rng.integers(-6, 7, (feats.shape[0], 1))).astype(np.float32)
    d2, _, L2 = oracle.pair_distances(feats * scale, offs, px, py)
    assert np.array_equal(d2, d) and np.array_equal(L2, L)
    # a generic positive rescaling moves FP32 inputs by rounding only
    scale = rng.uniform(0.1, 10.0, (feats.shape[0], 1)).astype(np.float32)
    d3, _, L3 = oracle.pair_distances(feats * scale, offs, px, py)
    assert np.max(np.abs(d3 - d)) < 1e-7


def test_mean_mode():
    rng = np.random.default_rng(6)
    dim = 40
    # single-frame items: mean mode equals DTW mode
    f = rng.standard_normal((6, dim)).astype(np.float32)
    offs = np.arange(7, dtype=np.int64)
    px, py = zip(*[(i, j) for i in range(6) for j in range(6)])
    dm, _, _ = oracle.pair_distances(f, offs, px, py, oracle.MODE_MEAN)
    dd, _, _ = oracle.pair_distances(f, offs, px, py, oracle.MODE_DTW)
    assert np.max(np.abs(dm - dd)) < 1e-15
    # mean of frames: two frames (1,0),(0,1) pool to (.5,.5), 45 degrees from (1,0)
    X = np.array([[1, 0], [0, 1], [1, 0]], dtype=np.float32)
    offs = np.array([0, 2, 3], dtype=np.int64)
    d, _, _ = oracle.pair_distances(X, offs, [0], [1], oracle.MODE_MEAN)
    assert abs(d[0] - 0.25) < 1e-15


# -------------------------------------------------------------------- cells

def _brute_triples(labels, on, by, across):
    n = labels.shape[0]
    out = set()
    for a, b, x in itertools.product(range(n), repeat=3):
        if a == x:
            continue
        if labels[a, on] != labels[x, on] or labels[b, on] == labels[a, on]:
            continue
        if any(labels[a, k] != labels[x, k] or labels[b, k] != labels[x, k] for k in by):
            continue
        if across is not None:
            if labels[a, across] != labels[b, across] or labels[x, across] == labels[a, across]:
                continue
        out.add((a, b, x))
    return out


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("task", [
    (0, (), None), (0, (1,), None), (0, (1, 2), None), (0, (1,), 2), (0, (), 2),
    (2, (1,), 0),
])
def test_cells_against_brute_force(seed, task):
    on, by, across = task
    rng = np.random.default_rng(seed)
    n = 26
    labels = np.stack([rng.integers(0, 3, n), rng.integers(0, 2, n), rng.integers(0, 3, n)],
                      axis=1)
    cells = oracle.enumerate_cells(labels, on, by, across)
    got = []
    for c in cells:
        assert c.P != c.Q
        for x in c.X:
            for a in c.A:
                if a != x:
                    for b in c.B:
                        got.append((a, b, x))
        # every triple of a cell carries the cell's key
        assert all(labels[i, on] == c.P for i in c.A + c.X)
        assert all(labels[i, on] == c.Q for i in c.B)
    assert len(got) == len(set(got))            # no triple in two cells
    assert set(got) == _brute_triples(labels, on, by, across)
    assert sum(c.count for c in cells) == len(got)


def test_within_cell_count_formula():
    # |C| = |P| (|P| - 1) |Q| in a within cell (a == x excluded)
    labels = np.array([[0, 0, 0]] * 4 + [[1, 0, 0]] * 3)
    cells = oracle.enumerate_cells(labels, 0, (1, 2), None)
    counts = {(c.P, c.Q): c.count for c in cells}
    assert counts == {(0, 1): 4 * 3 * 3, (1, 0): 3 * 2 * 4}


# ------------------------------------------------------------ cell scoring

def test_score_hand_example():
    # x, a, b from the DTW golden lines (a) and (b): d(x,a) = 0 < d(x,b) = .25
    X = _frames("1 0 ; 0 1")
    A = _frames("1 0 ; 1 0 ; 0 1")
    B = _frames("0 1 ; 0 1")
    feats = np.concatenate([X, A, B])
    offs = np.array([0, 2, 5, 7], dtype=np.int64)
    labels = np.array([[0, 0, 1], [0, 0, 0], [1, 0, 0]])   # x speaker 1, a/b speaker 0
    err, cells, scores, dd = oracle.abx_error(feats, offs, labels, on=0, by=(1,), across=2,
                                              levels=[(2,)])
    cell = [c for c in cells if c.P == 0 and c.across == (0, 1)][0]
    sc = scores[cells.index(cell)]
    assert dd[(0, 1)] == 0.0 and dd[(0, 2)] == 0.25
    assert sc == (2, 1)


def test_ties_score_half_and_swap_symmetry():
    rng = np.random.default_rng(7)
    # all items identical single frames: every comparison ties -> D_C = 1/2
    feats = np.tile(rng.standard_normal((1, 16)).astype(np.float32), (9, 1))
    offs = np.arange(10, dtype=np.int64)
    labels = np.stack([np.arange(9) % 3, np.zeros(9, int), np.zeros(9, int)], axis=1)
    err, cells, scores, _ = oracle.abx_error(feats, offs, labels, 0, (1,), None, [(1,)])
    assert all(s[0] == s[1] for s in scores) and err == 0.5
    # random items: swapping the roles of A and B gives 1 - D_C (no ties)
    w = synth.make_workload(40, 24, 3, 1, 1, 2, 6, "uniform", seed=8)
    cells = oracle.enumerate_cells(w.labels, 0, (1,), None)
    pairs = oracle.needed_pairs(cells)
    d, _, _ = oracle.pair_distances(w.feats, w.offsets, [p[0] for p in pairs],
                                    [p[1] for p in pairs])
    dd = {p: v for p, v in zip(pairs, d)}
    sc = oracle.score_cells(cells, dd)
    for c, (num2, cnt) in zip(cells, sc):
        if len(c.A) != len(c.B):
            continue
        # role swap: compare d(x, b) < d(x, a) on the same triples
        sw = 0
        for x in c.X:
            for a in c.A:
                if a == x:
                    continue
                for b in c.B:
                    sw += 2 * (dd[(x, b)] < dd[(x, a)]) + (dd[(x, b)] == dd[(x, a)])
        assert sw == 2 * cnt - num2


# ------------------------------------------------------------------ collapse

def test_collapse_golden():
    cells, scores, expects = [], [], []
    with open(os.path.join(GOLDEN, "collapse_handworked.txt")) as fh:
        for line in fh:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "cell":
                P, Q, ctx, spk, num2, cnt = map(int, t[1:])
                cells.append(oracle.Cell(P, Q, (ctx, spk), None))
                scores.append((num2, cnt))
            elif t[0] == "expect":
                expects.append((t[1], float(t[2])))
    names = {"context": 1, "speaker": 2}
    assert len(expects) == 3
    for spec, want in expects:
        if spec == "weighted":
            got = oracle.collapse(cells, scores, [], (1, 2), None, weighted=True)
        else:
            levels = [(names[s],) for s in spec.split(",")]
            got = oracle.collapse(cells, scores, levels, (1, 2), None)
        assert got == want, (spec, got)


def test_collapse_across_golden():
    """Across-speaker collapse: the speaker level averages over the ordered
    (s_ab, s_x) pairs jointly; a nested mean over s_x then s_ab (or the
    reverse) or a swapped level order gives another value."""
    from fractions import Fraction
    cells, scores, expects = [], [], []
    with open(os.path.join(GOLDEN, "collapse_across_handworked.txt")) as fh:
        for line in fh:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "cell":
                P, Q, ctx, s_ab, s_x, num2, cnt = map(int, t[1:])
                cells.append(oracle.Cell(P, Q, (ctx,), (s_ab, s_x)))
                scores.append((num2, cnt))
            elif t[0] == "expect":
                expects.append((t[1], Fraction(t[2])))
    names = {"context": 1, "speaker": 2}
    assert len(expects) == 3 and len(cells) == 7
    for spec, want in expects:
        if spec == "weighted":
            got = oracle.collapse(cells, scores, [], (1,), 2, weighted=True)
        else:
            levels = [(names[s],) for s in spec.split(",")]
            got = oracle.collapse(cells, scores, levels, (1,), 2)
        # the means are not dyadic: compare with the exact fraction to within
        # a few units of FP64 rounding
        assert abs(got - float(want)) < 1e-15, (spec, got, want)


# ---------------------------------------------------- Fig. 2 Gaussian setting

def test_gaussian_zero_shift_is_chance():
    w = synth.gaussian_2d(60, 0.0, seed=9)
    err, cells, scores, _ = oracle.abx_error(w.feats, w.offsets, w.labels, 0, (), None, [],
                                             weighted=True)
    # identical distributions: each (x, a, b) decision is a fair coin; the
    # std of the pooled estimate is far below 0.05 at this size
    assert abs(err - 0.5) < 0.05


def test_separated_classes_have_zero_error():
    # two classes with orthogonal means and small noise in 64-D
    rng = np.random.default_rng(10)
    mu = np.eye(64, dtype=np.float32)[:2] * 10
    lab = np.repeat([0, 1], 15)
    feats = (mu[lab] + 0.1 * rng.standard_normal((30, 64))).astype(np.float32)
    labels = np.stack([lab, np.zeros(30, int), np.zeros(30, int)], axis=1)
    offs = np.arange(31, dtype=np.int64)
    err, *_ = oracle.abx_error(feats, offs, labels, 0, (), None, [])
    assert err == 0.0


# ------------------------------------------------------- other distances

def test_other_distances_golden():
    kinds = {"cosine": oracle.COSINE, "euclidean": oracle.EUCLIDEAN, "kl": oracle.KL}
    n = 0
    with open(os.path.join(GOLDEN, "other_distances_handworked.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, u, v, want = line.split(";")
            got = oracle.distance(_frames(u)[0], _frames(v)[0], kinds[kind.strip()])
            assert abs(got - float(want)) < 1e-12, (line, got)
            n += 1
    assert n == 11


def test_other_distances_relations():
    rng = np.random.default_rng(11)
    for _ in range(50):
        u = rng.standard_normal(33).astype(np.float32)
        v = rng.standard_normal(33).astype(np.float32)
        ang = oracle.distance(u, v, oracle.ANGULAR)
        # cosine distance = 1 - cos(pi * angular)
        assert abs(oracle.distance(u, v, oracle.COSINE) - (1 - math.cos(math.pi * ang))) < 1e-12
        # Euclidean against numpy's norm of the difference (FP64)
        e = np.linalg.norm(u.astype(np.float64) - v.astype(np.float64))
        assert abs(oracle.distance(u, v, oracle.EUCLIDEAN) - e) < 1e-12
        # law of cosines links the Euclidean and cosine distances
        nu, nv = np.linalg.norm(u.astype(np.float64)), np.linalg.norm(v.astype(np.float64))
        c = 1 - oracle.distance(u, v, oracle.COSINE)
        assert abs(e * e - (nu * nu + nv * nv - 2 * nu * nv * c)) < 1e-9


def test_kl_distance_relations():
    """The symmetrised KL against scipy's elementwise relative entropy (an
    independent formula), and its invariants."""
    from scipy.special import rel_entr
    rng = np.random.default_rng(13)
    for _ in range(50):
        u = rng.uniform(0.01, 3.0, 17).astype(np.float32)
        v = rng.uniform(0.01, 3.0, 17).astype(np.float32)
        p = u.astype(np.float64) / u.astype(np.float64).sum()
        q = v.astype(np.float64) / v.astype(np.float64).sum()
        want = 0.5 * (rel_entr(p, q).sum() + rel_entr(q, p).sum())
        got = oracle.distance(u, v, oracle.KL)
        assert abs(got - want) < 1e-12 * max(1.0, want)
        assert got >= 0.0 and abs(got - oracle.distance(v, u, oracle.KL)) < 1e-15
        # a frame is a distribution up to scale
        assert abs(oracle.distance(4.0 * u, v, oracle.KL) - got) < 1e-12
        assert oracle.distance(u, 2.0 * u, oracle.KL) < 1e-15
    # undefined for a non-positive component
    assert math.isnan(oracle.distance(np.array([1, 0], np.float32),
                                      np.array([1, 1], np.float32), oracle.KL))
    assert math.isnan(oracle.distance(np.array([1, 1], np.float32),
                                      np.array([-1, 2], np.float32), oracle.KL))


def test_dtw_with_kl_distance():
    rng = np.random.default_rng(14)
    T = rng.integers(1, 6, 6)
    offs = np.concatenate([[0], np.cumsum(T)]).astype(np.int64)
    feats = rng.uniform(0.05, 2.0, (int(offs[-1]), 10)).astype(np.float32)
    px, py = zip(*[(i, j) for i in range(6) for j in range(6)])
    d, c, L = oracle.pair_distances(feats, offs, px, py, kind=oracle.KL)
    D = d.reshape(6, 6)
    assert np.allclose(np.diag(D), 0, atol=1e-12) and np.array_equal(D, D.T)
    for (i, j, dv) in zip(px, py, d):
        X = feats[offs[i]:offs[i + 1]]
        Y = feats[offs[j]:offs[j + 1]]
        m = np.array([[oracle.distance(a, b, oracle.KL) for b in Y] for a in X])
        cc, LL = oracle.dtw(m)
        assert abs(cc / LL - dv) < 1e-12
    # mean mode: KL of the frame means
    a, _, _ = oracle.pair_distances(feats, offs, px, py, oracle.MODE_MEAN, kind=oracle.KL)
    for (i, j, av) in zip(px, py, a):
        mx = feats[offs[i]:offs[i + 1]].astype(np.float64).mean(0)
        my = feats[offs[j]:offs[j + 1]].astype(np.float64).mean(0)
        p, q = mx / mx.sum(), my / my.sum()
        assert abs(av - 0.5 * np.sum((p - q) * (np.log(p) - np.log(q)))) < 1e-12


def test_dtw_with_other_distances():
    rng = np.random.default_rng(12)
    T = rng.integers(1, 7, 8)
    offs = np.concatenate([[0], np.cumsum(T)]).astype(np.int64)
    feats = rng.standard_normal((int(offs[-1]), 12)).astype(np.float32)
    px, py = zip(*[(i, j) for i in range(8) for j in range(8)])
    for kind in (oracle.COSINE, oracle.EUCLIDEAN):
        d, c, L = oracle.pair_distances(feats, offs, px, py, kind=kind)
        D = d.reshape(8, 8)
        assert np.allclose(np.diag(D), 0, atol=1e-6) and np.array_equal(D, D.T)
        # DTW over the distance matrix built one frame pair at a time
        for (i, j, dv) in zip(px, py, d):
            X = feats[offs[i]:offs[i + 1]]
            Y = feats[offs[j]:offs[j + 1]]
            m = np.array([[oracle.distance(a, b, kind) for b in Y] for a in X])
            cc, LL = oracle.dtw(m)
            assert abs(cc / LL - dv) < 1e-12
    # single frames: mean mode equals DTW mode for every distance
    f1 = rng.standard_normal((5, 9)).astype(np.float32)
    o1 = np.arange(6, dtype=np.int64)
    qx, qy = zip(*[(i, j) for i in range(5) for j in range(5)])
    for kind in (oracle.ANGULAR, oracle.COSINE, oracle.EUCLIDEAN):
        a, _, _ = oracle.pair_distances(f1, o1, qx, qy, oracle.MODE_MEAN, kind=kind)
        b, _, _ = oracle.pair_distances(f1, o1, qx, qy, oracle.MODE_DTW, kind=kind)
        assert np.max(np.abs(a - b)) < 1e-12
