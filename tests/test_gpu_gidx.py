"""Proximity-graph index (Sec. 5.4, graph-based non-exhaustive oracle) through the C-ABI
against the CPU oracle.

The graph (every point's M nearest others by (FP64 distance, id), made undirected) and
each query's traversal are exactly defined, so the GPU's adjacency and range sets must
equal the oracle's bit for bit; every returned point is a true member (no false
positives), and with a beam as wide as the data on a connected graph the rows are the
exact range sets.  Recall against the exact sets is reported, not pinned."""
import numpy as np
import pytest

import oracle
from paper_2601_01405_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bm():
    from paper_2601_01405_gb300 import _build, binding
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


@pytest.fixture(scope="module")
def data():
    return W.isotropic(12000, 16, 10, seed=91)


@pytest.fixture(scope="module")
def index(bm, data):
    return bm.GraphIndex(torch.from_numpy(data).cuda(), M=10, n_entries=32)


@pytest.fixture(scope="module")
def ref_graph(data):
    return oracle.graph_index(data, 10)


def test_graph_matches_oracle(index, ref_graph):
    off, adj = ref_graph
    assert np.array_equal(index.adj_off.cpu().numpy(), off)
    assert np.array_equal(index.adj.cpu().numpy(), adj)


@pytest.mark.parametrize("M,name", [(6, "tie"), (12, "mix"), (4, "roll")])
def test_graph_other_data(bm, M, name):
    X = {"tie": W.tiny_grid_cloud(3000, 3, 1, span=6, seed=92),
         "mix": W.make("mix32-n32k-d64")[:8000],
         "roll": W.make("roll-n50k-d128")[:6000]}[name]
    g = bm.GraphIndex(torch.from_numpy(np.ascontiguousarray(X)).cuda(), M=M, n_entries=16)
    off, adj = oracle.graph_index(X, M)
    assert np.array_equal(g.adj_off.cpu().numpy(), off) and np.array_equal(g.adj.cpu().numpy(), adj)


@pytest.mark.parametrize("ef,max_visits,eps", [(1, 4096, 3.0), (8, 4096, 3.0), (32, 4096, 3.0), (64, 200, 3.5),
                                               (16, 4096, 2.0)])
def test_range_query_matches_oracle(index, data, ref_graph, ef, max_visits, eps):
    Q = data[::41]
    off, ids, st = index.range_query(torch.from_numpy(Q).cuda(), eps, ef, max_visits)
    torch.cuda.synchronize()
    go, gi = oracle.graph_range_query(data, ref_graph[0], ref_graph[1], Q, eps, 32, ef, max_visits)
    assert np.array_equal(off.cpu().numpy(), go) and np.array_equal(ids.cpu().numpy(), gi)
    eo, ei = oracle.range_query(data, Q, eps)
    for j in range(Q.shape[0]):      # conservative: no false positives
        assert set(gi[go[j]:go[j + 1]].tolist()) <= set(ei[eo[j]:eo[j + 1]].tolist())
    if max_visits == 200:
        assert st["truncated"] == 1


def test_queries_off_the_points(index, data, ref_graph):
    Q = (data[::53] + W.isotropic(data[::53].shape[0], 16, 10, seed=93) * np.float32(0.25)).astype(np.float32)
    off, ids, st = index.range_query(torch.from_numpy(Q).cuda(), 3.0, 16)
    go, gi = oracle.graph_range_query(data, ref_graph[0], ref_graph[1], Q, 3.0, 32, 16, 4096)
    assert np.array_equal(off.cpu().numpy(), go) and np.array_equal(ids.cpu().numpy(), gi)


def test_wide_beam_is_exact(bm):
    X = W.isotropic(3000, 6, 10, seed=94)
    g = bm.GraphIndex(torch.from_numpy(X).cuda(), M=8, n_entries=1)
    Q = X[::17]
    off, ids, _ = g.range_query(torch.from_numpy(Q).cuda(), 1.4, 256, 3000)
    eo, ei = oracle.range_query(X, Q, 1.4)
    ro, ri = oracle.graph_range_query(X, g.adj_off.cpu().numpy(), g.adj.cpu().numpy(), Q, 1.4, 1, 256, 3000)
    assert np.array_equal(ids.cpu().numpy(), ri)
    if np.array_equal(ri, ei):       # the beam reached every ball in full
        assert np.array_equal(off.cpu().numpy(), eo)


def test_fixed_landmark_and_end_to_end_builds(bm, index, data, ref_graph):
    Xd = torch.from_numpy(data).cuda()
    exact = bm.bm_build(Xd, 3.0)
    lm = exact["landmarks"].cpu().numpy()
    fixed = index.build(3.0, 16, landmarks=exact["landmarks"])
    ro, ri = oracle.graph_range_query(data, ref_graph[0], ref_graph[1], data[lm], 3.0, 32, 16, 4096)
    assert np.array_equal(fixed["offsets"].cpu().numpy(), ro) and np.array_equal(fixed["ids"].cpu().numpy(), ri)
    e_ref = oracle.edges(data, lm, ro, ri, 3.0)
    assert np.array_equal(fixed["edges"].cpu().numpy(), e_ref)
    assert set(map(tuple, e_ref.tolist())) <= set(map(tuple, exact["edges"].cpu().numpy().tolist()))
    # end to end: the greedy driven by the graph's range sets
    out = index.build(3.0, 16)
    lm2 = out["landmarks"].cpu().numpy()
    assert np.all(np.diff(lm2) > 0)
    ro2, ri2 = oracle.graph_range_query(data, ref_graph[0], ref_graph[1], data[lm2], 3.0, 32, 16, 4096)
    assert np.array_equal(out["offsets"].cpu().numpy(), ro2) and np.array_equal(out["ids"].cpu().numpy(), ri2)
    n = data.shape[0]
    first_cover = np.full(n, n, dtype=np.int64)
    for k, l in enumerate(lm2):
        members = ri2[ro2[k]:ro2[k + 1]]
        first_cover[members] = np.minimum(first_cover[members], l)
    is_lm = np.zeros(n, bool)
    is_lm[lm2] = True
    assert np.array_equal(is_lm, ~(first_cover < np.arange(n)))
    assert np.array_equal(out["edges"].cpu().numpy(), oracle.edges(data, lm2, ro2, ri2, 3.0))


def test_errors(bm, index, data):
    Q = torch.from_numpy(data[:5]).cuda()
    for ef in (0, 257):
        with pytest.raises(bm.BallMapperError) as ei:
            index.range_query(Q, 1.0, ef)
        assert ei.value.status == bm.BM_ERR_ARG
    with pytest.raises(bm.BallMapperError):
        bm.GraphIndex(torch.from_numpy(data[:10]).cuda(), M=10)
