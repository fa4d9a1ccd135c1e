"""Checks that pin the CPU oracle to facts fixed by the paper and by mathematics.

Each ``pin_*`` raises AssertionError when the oracle disagrees.  They are used
by ``test_oracle_pins.py`` on the real oracle and by ``test_oracle_mutants.py``
on deliberately broken copies of it (every planted mistake must trip a pin).
"""
from __future__ import annotations

import json
import os

import numpy as np

import oracle
from oracle import brute
from paper_2601_01405_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def rows(offsets, ids):
    return [ids[offsets[i]:offsets[i + 1]].tolist() for i in range(len(offsets) - 1)]


def sqd(X, Y):
    """All-pairs FP64 squared distances by the direct formula (numpy broadcasting)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return ((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=2)


def _check_case(out, case):
    assert out["landmarks"].tolist() == case["landmarks"], ("landmarks", out["landmarks"], case)
    assert rows(out["offsets"], out["ids"]) == case["members"], ("members", case["eps"])
    assert out["edges"].tolist() == case["edges"], ("edges", out["edges"], case)


def pin_line():
    g = golden("line.json")
    for d in (1, 3):
        X = W.line_points(10, d)
        for case in g["cases"]:
            _check_case(oracle.build(X, case["eps"]), case)


def pin_grid():
    g = golden("grid.json")
    X = W.grid_points(3)
    for case in g["cases"]:
        _check_case(oracle.build(X, case["eps"]), case)


def pin_degenerate():
    # n = 0
    out = oracle.build(np.zeros((0, 3), dtype=np.float32), 1.0)
    assert out["landmarks"].size == 0 and out["edges"].size == 0 and out["offsets"].tolist() == [0]
    # n = 1
    out = oracle.build(np.ones((1, 4), dtype=np.float32), 0.5)
    assert out["landmarks"].tolist() == [0] and rows(out["offsets"], out["ids"]) == [[0]]
    # all points identical: one landmark, everyone a member (0 < eps), no edge
    X = np.full((7, 2), 0.25, dtype=np.float32)
    out = oracle.build(X, 1e-3)
    assert out["landmarks"].tolist() == [0]
    assert rows(out["offsets"], out["ids"]) == [list(range(7))]
    assert out["edges"].shape[0] == 0
    # eps larger than the diameter: a single ball holds everything
    X = W.isotropic(50, 3, 10, seed=5)
    out = oracle.build(X, 1e3)
    assert out["landmarks"].tolist() == [0] and out["ids"].tolist() == list(range(50))
    # d = 1, two far groups: two landmarks, no edge
    X = np.array([[0.0], [0.5], [10.0], [10.25]], dtype=np.float32)
    out = oracle.build(X, 1.0)
    assert out["landmarks"].tolist() == [0, 2]
    assert rows(out["offsets"], out["ids"]) == [[0, 1], [2, 3]]
    assert out["edges"].shape[0] == 0


def pin_brute(seeds=range(40)):
    """Tiny tie-heavy clouds against the exact rational brute force (brute.py)."""
    for s in seeds:
        rng = np.random.default_rng(1000 + s)
        n = int(rng.integers(1, 13))
        d = int(rng.integers(1, 4))
        k = 2
        X = W.tiny_grid_cloud(n, d, k, span=6, seed=s)
        eps = float(rng.choice([0.5, 0.75, 1.0, 1.25, 1.5, 2.0]))
        ref = brute.build(X, eps, k)
        out = oracle.build(X, eps)
        assert out["landmarks"].tolist() == ref["landmarks"], (s, "landmarks")
        assert rows(out["offsets"], out["ids"]) == ref["members"], (s, "members")
        assert [tuple(e) for e in out["edges"].tolist()] == ref["edges"], (s, "edges")


def pin_fixpoint(X, eps):
    """The index-order greedy result is the unique L with
    x in L  <=>  no l in L, l < x, has D(l, x) < eps^2."""
    lm = oracle.greedy(X, eps)
    D = sqd(X[lm], X)
    inside = D < oracle.eps_squared(eps)
    n = X.shape[0]
    is_lm = np.zeros(n, dtype=bool)
    is_lm[lm] = True
    earlier = lm[:, None] < np.arange(n)[None, :]
    covered_by_earlier = (inside & earlier).any(axis=0)
    assert np.array_equal(is_lm, ~covered_by_earlier)


def pin_invariants(X, eps):
    """eps-net (Def. 2.1 / rho-cover and alpha-separation, Sec. 5.1, Def. 5.4 and Thm. 5.5 with delta = 0),
    memberships equal to the full balls, CSR rows sorted and unique."""
    out = oracle.build(X, eps)
    lm, off, ids = out["landmarks"], out["offsets"], out["ids"]
    e2 = oracle.eps_squared(eps)
    assert np.all(np.diff(lm) > 0)
    D = sqd(X[lm], X)
    # membership = full open ball, in ascending id order
    for i in range(lm.size):
        assert ids[off[i]:off[i + 1]].tolist() == np.nonzero(D[i] < e2)[0].tolist()
    # cover: every point within eps of some landmark; landmarks are members of their own balls
    assert (D < e2).any(axis=0).all()
    # separation: distinct landmarks at squared distance >= eps^2
    DL = D[:, lm]
    np.fill_diagonal(DL, np.inf)
    assert (DL >= e2).all()
    return out


def pin_witness(X, eps):
    """Edge {i,j} exists iff the witness radius tau_ij < eps (Sec. 5.2, Def. 5.9):
    tau_ij^2 = min_x max(D(x,l_i), D(x,l_j))."""
    out = oracle.build(X, eps)
    lm = out["landmarks"]
    D = sqd(X[lm], X)
    e2 = oracle.eps_squared(eps)
    L = lm.size
    expect = []
    for i in range(L):
        tau2 = np.maximum(D[i][None, :], D[i + 1:]).min(axis=1) if i + 1 < L else np.zeros(0)
        for off, t in enumerate(tau2):
            if t < e2:
                expect.append((i, i + 1 + off))
    assert [tuple(e) for e in out["edges"].tolist()] == expect


def pin_prune(X, eps):
    out = oracle.build(X, eps, prune=True)
    e0 = oracle.edges(X, out["landmarks"], out["offsets"], out["ids"], eps, prune=False)
    assert np.array_equal(out["edges"], e0)


def pin_balltree(X, eps, Q=None):
    """An exact accelerated range query preserves every range set (Sec. 3.1 ball tree
    against the Sec. 5 (Def. 5.1) full scan)."""
    if Q is None:
        Q = X[oracle.greedy(X, eps)]
    bt = oracle.BallTree(X, leaf_size=40)
    o1, i1 = bt.range_query(Q, eps)
    o2, i2 = oracle.range_query(X, Q, eps)
    assert np.array_equal(o1, o2) and np.array_equal(i1, i2)
    assert bt.node_count > 1 or X.shape[0] <= 40


def pin_knn_scipy(X, k):
    """k-th NN distance (self counted first) against scipy's kd-tree."""
    from scipy.spatial import cKDTree
    ref = cKDTree(np.asarray(X, dtype=np.float64)).query(np.asarray(X, dtype=np.float64), k=k)[0][:, -1]
    got = oracle.kth_nn_dist(X, k)
    assert np.allclose(got, ref, rtol=1e-12, atol=0.0)


def pin_range_scipy(X, Q, eps):
    """Range sets on continuous (tie-free) data against scipy's kd-tree ball query.
    scipy's ball is closed; with no point at distance exactly eps it equals the open ball."""
    from scipy.spatial import cKDTree
    X64 = np.asarray(X, dtype=np.float64)
    Q64 = np.asarray(Q, dtype=np.float64)
    D = np.sqrt(sqd(Q64, X64))
    assert not np.any(np.abs(D - eps) < 1e-9), "data has a near-tie; choose another eps"
    ref = cKDTree(X64).query_ball_point(Q64, r=eps)
    off, ids = oracle.range_query(X64, Q64, eps)
    for j in range(Q64.shape[0]):
        assert ids[off[j]:off[j + 1]].tolist() == sorted(ref[j])


def pin_pair_sqdist(X, Q, k):
    """Squared distances of listed (query row, point) pairs, with Q and X different sets
    of different sizes, equal the exact rational values: coordinates are multiples of
    2^-k, so D = sum_i (m_q,i - m_x,i)^2 / 4^k with integer m, and FP64 holds it
    exactly.  Indices stay below both row counts, so a swap of the two roles reads
    valid rows of the other set and shows as wrong values."""
    from fractions import Fraction
    assert X.shape[0] != Q.shape[0]
    rng = np.random.default_rng(3)
    lim = min(X.shape[0], Q.shape[0])
    qrow = rng.integers(0, lim, 200)
    xcol = rng.integers(0, lim, 200)
    got = oracle.pair_sqdist(X, Q, qrow, xcol)
    scale = 2 ** k
    for t in range(qrow.size):
        mq = [int(Fraction(float(v)) * scale) for v in Q[qrow[t]]]
        mx = [int(Fraction(float(v)) * scale) for v in X[xcol[t]]]
        exact = Fraction(sum((a - b) ** 2 for a, b in zip(mq, mx)), 4 ** k)
        assert Fraction(float(got[t])) == exact, t


def pin_paper():
    g = golden("paper_gaussian.json")
    X = W.paper_gaussian_fp64(g["n"], g["d"], seed=0)
    eps = oracle.occupancy_eps(X, g["k"])
    assert abs(eps - g["eps_printed"]) < g["eps_tolerance"], eps
    out = oracle.build(X, eps)
    assert out["landmarks"].size == g["landmarks"]
    assert out["edges"].shape[0] == g["edges"]


def pin_masked():
    """Verified range set over probed cells (Sec. 5.3): with every cell probed it is the
    exact range set; in general it equals the exact set filtered by cell membership."""
    X = W.isotropic(1500, 6, 10, seed=12)
    Q = X[:40]
    rng = np.random.default_rng(4)
    cell = rng.integers(0, 12, X.shape[0]).astype(np.int32)
    allp = np.tile(np.arange(12, dtype=np.int32), (Q.shape[0], 1))
    o1, i1 = oracle.masked_range_query(X, Q, 2.0, cell, 12, allp)
    o2, i2 = oracle.range_query(X, Q, 2.0)
    assert np.array_equal(o1, o2) and np.array_equal(i1, i2)
    probes = np.stack([rng.choice(12, 3, replace=False) for _ in range(Q.shape[0])]).astype(np.int32)
    o3, i3 = oracle.masked_range_query(X, Q, 2.0, cell, 12, probes)
    for j in range(Q.shape[0]):
        full = i2[o2[j]:o2[j + 1]]
        keep = full[np.isin(cell[full], probes[j])]
        assert i3[o3[j]:o3[j + 1]].tolist() == keep.tolist()


# ---------------------------------------------------------------- farthest point sampling
def _fps_points(name):
    return W.line_points(10) if name == "line" else W.grid_points(3)


def pin_fps_golden():
    g = golden("fps_line.json")
    for case in g["cases"]:
        X = _fps_points(case["points"])
        out = oracle.fps_build(X, case["eps"], case["first"])
        _check_case(out, case)


def pin_fps_invariants(X, eps, first=0):
    """Sec. 2.2 / Def. 2.1 with open balls: the landmarks start at `first`, are pairwise at
    squared distance >= eps^2, every point lies in some open ball, and the selection
    distances (to the landmarks before) never increase."""
    lm = oracle.fps(X, eps, first)
    e2 = oracle.eps_squared(eps)
    assert lm[0] == first and np.unique(lm).size == lm.size
    D = sqd(X[lm], X)
    assert np.all(D.min(axis=0) < e2)                                 # cover
    DL = sqd(X[lm], X[lm])
    np.fill_diagonal(DL, np.inf)
    assert np.all(DL >= e2)                                            # separation
    sel = [DL[i, :i].min() for i in range(1, lm.size)]
    assert all(a >= b for a, b in zip(sel, sel[1:]))                   # non-increasing
    # the point after the last landmark would be closer than eps
    assert D.min(axis=0).max() < e2


def pin_fps_brute(seeds=range(12)):
    for seed in seeds:
        rng = np.random.default_rng(seed)
        n = int(rng.integers(1, 12))
        d = int(rng.integers(1, 4))
        X = W.tiny_grid_cloud(n, d, 1, span=4, seed=seed)
        eps = float(rng.choice([0.5, 1.0, 1.5, 2.0]))
        first = int(rng.integers(0, n))
        assert oracle.fps(X, eps, first).tolist() == brute.fps(X, eps, 1, first), (seed, n, d, eps)


# ---------------------------------------------------------------- coloring
def pin_color_golden():
    g = golden("color_line.json")
    X = W.line_points(10)
    out = oracle.build(X, g["eps"])
    f = X[:, 0].astype(np.float64) ** 2
    for stat in ("mean", "median", "min", "max"):
        got = oracle.color(out["offsets"], out["ids"], f, stat)
        assert got.tolist() == g[stat], (stat, got)


def pin_color_lipschitz(X, eps, k=2.5, seed=0):
    """Sec. 2.3 with f = k <w, x>, |w| = 1 (k-Lipschitz) and a coloring between the
    ball's minimum and maximum of f (mean, median, min, max):
      |c(l_i) - f(l_i)| < k eps                 (every member is within eps of l_i)
      max_{x in X_i} |f(x) - c(l_i)| < 2 k eps  (the ball's diameter is below 2 eps)
      |c(l_i) - c(l_j)| < 4 k eps on every edge (a shared point links the two)
    The paper states the second bound as k eps and the third as 2 k eps; those do not
    follow (a lopsided ball breaks them for the mean), these do."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(X.shape[1])
    w /= np.linalg.norm(w)
    f = k * (np.asarray(X, dtype=np.float64) @ w)
    out = oracle.build(X, eps)
    lm, off, ids, E = out["landmarks"], out["offsets"], out["ids"], out["edges"]
    slack = 1e-9 * k * eps
    for stat in ("mean", "median", "min", "max"):
        c = oracle.color(off, ids, f, stat)
        for i in range(lm.size):
            row = f[ids[off[i]:off[i + 1]]]
            assert row.min() <= c[i] <= row.max(), (stat, i)
            assert abs(c[i] - f[lm[i]]) < k * eps + slack
            assert np.abs(row - c[i]).max() < 2 * k * eps + slack
        if E.size:
            assert np.abs(c[E[:, 0]] - c[E[:, 1]]).max() < 4 * k * eps + slack


def pin_color_values(X, eps, seed=1):
    """Each statistic against its definition on every row: the median is a middle value of
    the sorted row (or the mean of the two), min and max are attained, and a constant f
    colors every ball with that constant."""
    rng = np.random.default_rng(seed)
    out = oracle.build(X, eps)
    off, ids = out["offsets"], out["ids"]
    f = rng.standard_normal(X.shape[0])
    med = oracle.color(off, ids, f, "median")
    mn = oracle.color(off, ids, f, "min")
    mx = oracle.color(off, ids, f, "max")
    mean = oracle.color(off, ids, f, "mean")
    for i in range(off.size - 1):
        row = np.sort(f[ids[off[i]:off[i + 1]]])
        m = row.size
        assert med[i] == (row[m // 2] if m % 2 else (row[m // 2 - 1] + row[m // 2]) / 2.0)
        assert mn[i] == row[0] and mx[i] == row[-1]
        assert abs(mean[i] - row.sum() / m) <= 1e-12 * max(1.0, np.abs(row).sum())
    const = oracle.color(off, ids, np.full(X.shape[0], 3.25), "mean")
    assert np.all(const == 3.25)


# ---------------------------------------------------------------- graph-based range oracle
def pin_graph_golden():
    g = golden("graph_line.json")
    for case in g["cases"]:
        X = np.array(case["points"], dtype=np.float32)
        if "arcs" in case:
            assert oracle.knn_graph(X, case["M"]).tolist() == case["arcs"]
        off, adj = oracle.graph_index(X, case["M"])
        assert off.tolist() == case["adj_off"] and adj.tolist() == case["adj"], case
        Q = np.array(case["queries"], dtype=np.float32)
        ro, ri = oracle.graph_range_query(X, off, adj, Q, case["eps"], case["E"], case["ef"], case["max_visits"])
        assert rows(ro, ri) == case["rows"], (rows(ro, ri), case)


def pin_knn_graph_scipy(X, M):
    """M nearest other points on tie-free data, against scipy's k-d tree."""
    from scipy.spatial import cKDTree
    X64 = np.asarray(X, dtype=np.float64)
    ref = cKDTree(X64).query(X64, k=M + 1)[1][:, 1:]
    assert np.array_equal(oracle.knn_graph(X, M), ref)


def pin_graph_exhaustive_and_conservative(X, Q, eps, M=6):
    """With a beam as wide as the data and a connected graph every point is visited, so
    the rows are the exact range sets; with a narrow beam they stay subsets of them."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    off, adj = oracle.graph_index(X, M)
    n = X.shape[0]
    g = csr_matrix((np.ones(adj.size), adj, off), shape=(n, n))
    assert connected_components(g, directed=False)[0] == 1
    eo, ei = oracle.range_query(X, Q, eps)
    go, gi = oracle.graph_range_query(X, off, adj, Q, eps, 1, n, n)
    assert np.array_equal(go, eo) and np.array_equal(gi, ei)
    lo, li = oracle.graph_range_query(X, off, adj, Q, eps, 4, 2, n)
    for j in range(Q.shape[0]):
        assert set(li[lo[j]:lo[j + 1]].tolist()) <= set(ei[eo[j]:eo[j + 1]].tolist())
