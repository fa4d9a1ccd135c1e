"""CPU oracle for exact Ball Mapper construction -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it.

The arithmetic lives in ``bm_oracle.c`` (plain FP64 loops, one per definition
of the paper); this module compiles it with gcc, loads it with ctypes and
marshals numpy arrays.  ``brute.py`` is a second, differently written brute
force (exact integer/rational arithmetic) used to pin this one.

Functions and the passages they follow:
  greedy             Sec. 2.2 greedy epsilon-net, smallest uncovered index first
  range_query        Sec. 5 (Def. 5.1) exact range set R_r(q) = {x : d(q,x) < r}, full scan
  memberships        Sec. 2.3 X_i = X intersect B(l_i, eps), full balls
  edges              Sec. 2.1 nerve / Sec. 5.2 G_r(L): edge iff X_i, X_j intersect
  build              all of the above in order
  kth_nn_dist        Sec. 6.1 target-occupancy rule (self counted first)
  masked_range_query Sec. 5.3 verified range set over a candidate set (points of probed cells)
  BallTree           Sec. 3.1 ball tree construction and pruned range query
  fps                Sec. 2.2 farthest point sampling epsilon-net
  fps_build          the Ball Mapper on the farthest-point landmarks (memberships, edges)
  color              Sec. 2.3 coloring: mean / median / min / max of f over each ball
  knn_graph          M nearest other points of every point (the proximity graph's arcs)
  graph_index        undirected proximity graph (CSR), the graph-based index of Sec. 5.4
  graph_range_query  Sec. 5.4 partial graph traversal + exact decision (conservative range sets)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libbm_oracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def compile_library(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the oracle shared library with gcc (OpenMP, no FMA contraction)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def load_library(path: str):
    """Load a compiled oracle library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    lib.bmo_greedy.restype = ctypes.c_int64
    lib.bmo_greedy.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, _i32p]
    lib.bmo_range_count.restype = None
    lib.bmo_range_count.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, _f64p, ctypes.c_int64,
                                    ctypes.c_double, _i64p]
    lib.bmo_range_fill.restype = None
    lib.bmo_range_fill.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, _f64p, ctypes.c_int64,
                                   ctypes.c_double, _i64p, _i32p]
    lib.bmo_pair_sqdist.restype = None
    lib.bmo_pair_sqdist.argtypes = [_f64p, ctypes.c_int, _f64p, ctypes.c_int64, _i32p, _i32p, _f64p]
    lib.bmo_edges.restype = None
    lib.bmo_edges.argtypes = [_f64p, ctypes.c_int, _i32p, ctypes.c_int64, ctypes.c_double,
                              _i64p, _i32p, ctypes.c_int, _i64p, _i64p, _i32p]
    lib.bmo_kth_nn_dist.restype = ctypes.c_int
    lib.bmo_kth_nn_dist.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, _f64p]
    lib.bmo_bt_build.restype = ctypes.c_void_p
    lib.bmo_bt_build.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int]
    lib.bmo_bt_free.restype = None
    lib.bmo_bt_free.argtypes = [ctypes.c_void_p]
    lib.bmo_bt_node_count.restype = ctypes.c_int64
    lib.bmo_bt_node_count.argtypes = [ctypes.c_void_p]
    lib.bmo_bt_range_count.restype = ctypes.c_int
    lib.bmo_bt_range_count.argtypes = [ctypes.c_void_p, _f64p, ctypes.c_int64, ctypes.c_double, _i64p]
    lib.bmo_bt_range_fill.restype = ctypes.c_int
    lib.bmo_bt_range_fill.argtypes = [ctypes.c_void_p, _f64p, ctypes.c_int64, ctypes.c_double,
                                      _i64p, _i32p]
    lib.bmo_masked_range_count.restype = ctypes.c_int
    lib.bmo_masked_range_count.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, _f64p, ctypes.c_int64,
                                           ctypes.c_double, _i32p, ctypes.c_int, _i32p, ctypes.c_int, _i64p]
    lib.bmo_masked_range_fill.restype = ctypes.c_int
    lib.bmo_masked_range_fill.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, _f64p, ctypes.c_int64,
                                          ctypes.c_double, _i32p, ctypes.c_int, _i32p, ctypes.c_int, _i64p, _i32p]
    lib.bmo_fps.restype = ctypes.c_int64
    lib.bmo_fps.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int64, _i32p]
    lib.bmo_color.restype = ctypes.c_int
    lib.bmo_color.argtypes = [_i64p, _i32p, ctypes.c_int64, _f64p, ctypes.c_int, _f64p]
    lib.bmo_knn_graph.restype = ctypes.c_int
    lib.bmo_knn_graph.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _i32p]
    lib.bmo_graph_range.restype = ctypes.c_int
    lib.bmo_graph_range.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, _i64p, _i32p, _f64p, ctypes.c_int64,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _i64p, _i64p, _i32p]
    lib.bmo_num_threads.restype = ctypes.c_int
    lib.bmo_num_threads.argtypes = []
    lib.bmo_set_num_threads.restype = None
    lib.bmo_set_num_threads.argtypes = [ctypes.c_int]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(compile_library())
        return _lib


def _f64(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a), dtype=np.float64)
    if a.ndim == 1:
        a = a.reshape(1, -1) if a.size else a.reshape(0, 1)
    return a


def _ptr(a, t):
    return a.ctypes.data_as(t)


def eps_squared(eps) -> float:
    """eps^2 in FP64.  For a float32 eps the product is exact (24 x 24 bits < 53)."""
    e = float(eps)
    return e * e


def num_threads() -> int:
    return int(_load().bmo_num_threads())


def set_num_threads(t: int) -> None:
    _load().bmo_set_num_threads(int(t))


def greedy(X, eps) -> np.ndarray:
    """Landmark ids in greedy selection order (Sec. 2.2)."""
    X = _f64(X)
    n, d = X.shape
    out = np.empty(max(n, 1), dtype=np.int32)
    L = _load().bmo_greedy(_ptr(X, _f64p), n, d, eps_squared(eps), _ptr(out, _i32p))
    if L < 0:
        raise MemoryError("oracle greedy: allocation failed")
    return out[:L].copy()


def range_query(X, Q, eps):
    """CSR (offsets int64 [m+1], ids int32) with row j = {i : D(X_i, Q_j) < eps^2}."""
    X = _f64(X)
    Q = _f64(Q)
    n, d = X.shape
    m = Q.shape[0]
    if m and Q.shape[1] != d:
        raise ValueError("dimension mismatch")
    lib = _load()
    counts = np.zeros(m, dtype=np.int64)
    e2 = eps_squared(eps)
    if m:
        lib.bmo_range_count(_ptr(X, _f64p), n, d, _ptr(Q, _f64p), m, e2, _ptr(counts, _i64p))
    offsets = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    ids = np.empty(max(int(offsets[-1]), 1), dtype=np.int32)
    if m:
        lib.bmo_range_fill(_ptr(X, _f64p), n, d, _ptr(Q, _f64p), m, e2, _ptr(offsets, _i64p),
                           _ptr(ids, _i32p))
    return offsets, ids[: int(offsets[-1])].copy()


def masked_range_query(X, Q, eps, cell_of, nlist, probes):
    """Verified range set over probed cells (Sec. 5.3): row j = {i : cell_of[i] in
    probes[j], D(X_i, Q_j) < eps^2}, ascending.  probes: (m, nprobe) int32."""
    X = _f64(X)
    Q = _f64(Q)
    n, d = X.shape
    m = Q.shape[0]
    cell_of = np.ascontiguousarray(cell_of, dtype=np.int32)
    probes = np.ascontiguousarray(probes, dtype=np.int32).reshape(m, -1)
    nprobe = probes.shape[1]
    lib = _load()
    counts = np.zeros(max(m, 1), dtype=np.int64)
    e2 = eps_squared(eps)
    if m and lib.bmo_masked_range_count(_ptr(X, _f64p), n, d, _ptr(Q, _f64p), m, e2, _ptr(cell_of, _i32p),
                                        int(nlist), _ptr(probes, _i32p), nprobe, _ptr(counts, _i64p)):
        raise MemoryError("masked range query")
    offsets = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts[:m], out=offsets[1:])
    ids = np.empty(max(int(offsets[-1]), 1), dtype=np.int32)
    if m and lib.bmo_masked_range_fill(_ptr(X, _f64p), n, d, _ptr(Q, _f64p), m, e2, _ptr(cell_of, _i32p),
                                       int(nlist), _ptr(probes, _i32p), nprobe, _ptr(offsets, _i64p),
                                       _ptr(ids, _i32p)):
        raise MemoryError("masked range query")
    return offsets, ids[: int(offsets[-1])].copy()


def memberships(X, landmarks, eps):
    """Full ball of every landmark (Sec. 2.3), CSR in landmark order."""
    X = _f64(X)
    lm = np.asarray(landmarks, dtype=np.int64)
    Q = X[lm] if lm.size else np.zeros((0, X.shape[1]))
    return range_query(X, Q, eps)


def pair_sqdist(X, Q, qrow, xcol) -> np.ndarray:
    """D(Q[qrow[k]], X[xcol[k]]) in FP64 for listed pairs."""
    X = _f64(X)
    Q = _f64(Q)
    qrow = np.ascontiguousarray(qrow, dtype=np.int32)
    xcol = np.ascontiguousarray(xcol, dtype=np.int32)
    out = np.empty(qrow.size, dtype=np.float64)
    if qrow.size:
        _load().bmo_pair_sqdist(_ptr(X, _f64p), X.shape[1], _ptr(Q, _f64p), qrow.size,
                                _ptr(qrow, _i32p), _ptr(xcol, _i32p), _ptr(out, _f64p))
    return out


def edges(X, landmarks, offsets, ids, eps, prune: bool = True) -> np.ndarray:
    """Nerve 1-skeleton as an (E, 2) int32 array of landmark ordinals, i < j,
    lexicographic: {i, j} is an edge iff membership rows i and j intersect."""
    X = _f64(X)
    lm = np.ascontiguousarray(landmarks, dtype=np.int32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    if ids.size == 0:
        ids = np.zeros(1, dtype=np.int32)
    L = lm.size
    lib = _load()
    counts = np.zeros(max(L, 1), dtype=np.int64)
    if L:
        lib.bmo_edges(_ptr(X, _f64p), X.shape[1], _ptr(lm, _i32p), L, eps_squared(eps),
                      _ptr(offsets, _i64p), _ptr(ids, _i32p), int(prune), _ptr(counts, _i64p),
                      None, None)
    row_off = np.zeros(L + 1, dtype=np.int64)
    np.cumsum(counts[:L], out=row_off[1:])
    E = int(row_off[-1])
    out = np.empty((max(E, 1), 2), dtype=np.int32)
    if E:
        lib.bmo_edges(_ptr(X, _f64p), X.shape[1], _ptr(lm, _i32p), L, eps_squared(eps),
                      _ptr(offsets, _i64p), _ptr(ids, _i32p), int(prune), None,
                      _ptr(row_off, _i64p), _ptr(out, _i32p))
    return out[:E].copy()


def build(X, eps, prune: bool = True) -> dict:
    """Exact Ball Mapper: greedy landmarks, full-ball CSR memberships, nerve edges."""
    lm = greedy(X, eps)
    offsets, ids = memberships(X, lm, eps)
    e = edges(X, lm, offsets, ids, eps, prune=prune)
    return {"landmarks": lm, "offsets": offsets, "ids": ids, "edges": e}


def fps(X, eps, first: int = 0) -> np.ndarray:
    """Farthest-point landmarks in selection order (Sec. 2.2), starting at `first`."""
    X = _f64(X)
    n, d = X.shape
    out = np.empty(max(n, 1), dtype=np.int32)
    if not 0 <= first < max(n, 1):
        raise ValueError("first out of range")
    L = _load().bmo_fps(_ptr(X, _f64p), n, d, eps_squared(eps), int(first), _ptr(out, _i32p))
    if L < 0:
        raise MemoryError("oracle fps: allocation failed")
    return out[:L].copy()


def fps_build(X, eps, first: int = 0, prune: bool = True) -> dict:
    """Ball Mapper on the farthest-point landmarks: full-ball memberships and nerve edges
    in landmark selection order."""
    lm = fps(X, eps, first)
    offsets, ids = memberships(X, lm, eps)
    e = edges(X, lm, offsets, ids, eps, prune=prune)
    return {"landmarks": lm, "offsets": offsets, "ids": ids, "edges": e}


COLOR_STATS = {"mean": 0, "median": 1, "min": 2, "max": 3}


def color(offsets, ids, f, stat: str = "mean") -> np.ndarray:
    """c(l_i) = stat of f over CSR row i (Sec. 2.3); NaN for an empty row."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    if ids.size == 0:
        ids = np.zeros(1, dtype=np.int32)
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).ravel())
    rows = offsets.size - 1
    out = np.empty(max(rows, 1), dtype=np.float64)
    if rows and _load().bmo_color(_ptr(offsets, _i64p), _ptr(ids, _i32p), rows, _ptr(f, _f64p),
                                  COLOR_STATS[stat], _ptr(out, _f64p)):
        raise MemoryError("oracle color: allocation failed")
    return out[:rows].copy()


def knn_graph(X, M: int) -> np.ndarray:
    """(n, M) int32: the M nearest other points of every point, by (FP64 D, id)."""
    X = _f64(X)
    n, d = X.shape
    out = np.empty((max(n, 1), M), dtype=np.int32)
    if _load().bmo_knn_graph(_ptr(X, _f64p), n, d, int(M), _ptr(out, _i32p)):
        raise ValueError("knn_graph: M out of range or allocation failure")
    return out[:n].copy()


def graph_index(X, M: int):
    """Undirected proximity graph: the union of every point's M-nearest arcs and their
    reverses, as CSR (adj_off int64 [n+1], adj int32) with ascending neighbour lists."""
    nbr = knn_graph(X, M)
    n = nbr.shape[0]
    src = np.repeat(np.arange(n, dtype=np.int64), M)
    dst = nbr.astype(np.int64).ravel()
    keys = np.unique(np.concatenate([src * n + dst, dst * n + src]))
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, keys // n + 1, 1)
    return np.cumsum(off), (keys % n).astype(np.int32)


def graph_range_query(X, adj_off, adj, Q, eps, E: int, ef: int, max_visits: int):
    """Conservative range sets through the proximity graph (Sec. 5.4): CSR over the rows
    of Q of the visited points with D < eps^2 (entry, beam of ef, range expansion)."""
    X = _f64(X)
    Q = _f64(Q)
    n, d = X.shape
    m = Q.shape[0]
    adj_off = np.ascontiguousarray(adj_off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    if adj.size == 0:
        adj = np.zeros(1, dtype=np.int32)
    lib = _load()
    counts = np.zeros(max(m, 1), dtype=np.int64)
    e2 = eps_squared(eps)
    if m and lib.bmo_graph_range(_ptr(X, _f64p), n, d, _ptr(adj_off, _i64p), _ptr(adj, _i32p), _ptr(Q, _f64p), m, e2,
                                 int(E), int(ef), int(max_visits), _ptr(counts, _i64p), None, None):
        raise ValueError("graph range query failed")
    offsets = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts[:m], out=offsets[1:])
    ids = np.empty(max(int(offsets[-1]), 1), dtype=np.int32)
    if m and lib.bmo_graph_range(_ptr(X, _f64p), n, d, _ptr(adj_off, _i64p), _ptr(adj, _i32p), _ptr(Q, _f64p), m,
                                 e2, int(E), int(ef), int(max_visits), None, _ptr(offsets, _i64p), _ptr(ids, _i32p)):
        raise ValueError("graph range query failed")
    return offsets, ids[: int(offsets[-1])].copy()


def kth_nn_dist(X, k: int) -> np.ndarray:
    """Distance from each point to its k-th nearest neighbour, itself counted first."""
    X = _f64(X)
    n, d = X.shape
    out = np.empty(n, dtype=np.float64)
    rc = _load().bmo_kth_nn_dist(_ptr(X, _f64p), n, d, int(k), _ptr(out, _f64p))
    if rc != 0:
        raise ValueError("kth_nn_dist failed (k out of range or allocation failure)")
    return out


def occupancy_eps(X, k: int) -> float:
    """Target-occupancy scale (Sec. 6.1): median over points of the k-th NN distance.
    An even count takes the mean of the two middle values."""
    return float(np.median(kth_nn_dist(X, k)))


class BallTree:
    """Independent exact range oracle through the ball tree of Sec. 3.1."""

    def __init__(self, X, leaf_size: int = 40):
        self._X = _f64(X)
        n, d = self._X.shape
        self._d = d
        self._h = _load().bmo_bt_build(_ptr(self._X, _f64p), n, d, int(leaf_size))
        if not self._h:
            raise MemoryError("ball tree build failed")

    @property
    def node_count(self) -> int:
        return int(_load().bmo_bt_node_count(self._h))

    def range_query(self, Q, eps):
        Q = _f64(Q)
        m = Q.shape[0]
        lib = _load()
        counts = np.zeros(max(m, 1), dtype=np.int64)
        if m and lib.bmo_bt_range_count(self._h, _ptr(Q, _f64p), m, float(eps), _ptr(counts, _i64p)):
            raise RuntimeError("ball tree query failed")
        offsets = np.zeros(m + 1, dtype=np.int64)
        np.cumsum(counts[:m], out=offsets[1:])
        ids = np.empty(max(int(offsets[-1]), 1), dtype=np.int32)
        if m and lib.bmo_bt_range_fill(self._h, _ptr(Q, _f64p), m, float(eps), _ptr(offsets, _i64p),
                                       _ptr(ids, _i32p)):
            raise RuntimeError("ball tree query failed")
        return offsets, ids[: int(offsets[-1])].copy()

    def close(self):
        if self._h:
            _load().bmo_bt_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
