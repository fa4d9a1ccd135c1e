"""Inverted-file range queries (Sec. 5.3-5.4) through the C-ABI against the CPU oracle.

The index's cells and each query's probed cells come from heuristics (k-means,
nearest centroids); given them, the range sets are exactly defined -- the
verified range set over the probed cells -- and must match the oracle bit for
bit.  The heuristics themselves are checked through their defining properties."""
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
    return W.isotropic(20000, 32, 10, seed=41)


@pytest.fixture(scope="module")
def index(bm, data):
    return bm.IvfIndex(torch.from_numpy(data).cuda(), nlist=64, iters=10, sample=8192, seed=5)


def sqd(A, B):
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    return (A * A).sum(1)[:, None] + (B * B).sum(1)[None, :] - 2 * A @ B.T


def test_cells_are_nearest_centroids(index, data):
    cent = index.centroids.cpu().numpy()
    cell = index.cell_of.cpu().numpy()
    D = sqd(data, cent)
    tol = 1e-4 * (np.abs(D).max() + 1.0)
    assert np.all(D[np.arange(data.shape[0]), cell] <= D.min(1) + tol)
    assert np.bincount(cell, minlength=64).min() >= 1


@pytest.mark.parametrize("path", ["tc", "fp32"])
@pytest.mark.parametrize("nprobe", [1, 4, 17, 64])
def test_range_query_matches_masked_oracle(index, data, nprobe, path):
    """Both scans (the tensor-core tiles over cells laid out in whole tiles, and the FP32
    CUDA-core tiles) give the verified range set over the probed cells."""
    Q = data[::37]
    off, ids, probes, st = index.range_query(torch.from_numpy(Q).cuda(), 4.0, nprobe, path=path)
    p = probes.cpu().numpy()
    # probes: nprobe distinct cells, the nearest ones (up to float32 ties)
    D = sqd(Q, index.centroids.cpu().numpy())
    tol = 1e-4 * (np.abs(D).max() + 1.0)
    kth = np.sort(D, axis=1)[:, nprobe - 1]
    assert all(len(set(r)) == nprobe for r in p.tolist())
    assert np.all(D[np.arange(Q.shape[0])[:, None], p] <= kth[:, None] + tol)
    ro, ri = oracle.masked_range_query(data, Q, 4.0, index.cell_of.cpu().numpy(), 64, p)
    assert np.array_equal(off.cpu().numpy(), ro) and np.array_equal(ids.cpu().numpy(), ri)
    if nprobe == 64:   # every cell probed: the exact range set
        eo, ei = oracle.range_query(data, Q, 4.0)
        assert np.array_equal(ro, eo) and np.array_equal(ri, ei)


@pytest.mark.parametrize("path", ["tc", "fp32"])
def test_fixed_landmark_build(bm, index, data, path):
    """Fixed-landmark mode (Sec. 6.2): balls through the index, nerve of those balls;
    conservative, so every membership and edge is also exact (Prop. 5.15)."""
    Xd = torch.from_numpy(data).cuda()
    exact = bm.bm_build(Xd, 4.0)
    approx = index.build(4.0, 8, landmarks=exact["landmarks"], path=path)
    lm = exact["landmarks"].cpu().numpy()
    _, _, probes, _ = index.range_query(torch.from_numpy(data[lm]).cuda(), 4.0, 8)
    ro, ri = oracle.masked_range_query(data, data[lm], 4.0, index.cell_of.cpu().numpy(), 64, probes.cpu().numpy())
    assert np.array_equal(approx["offsets"].cpu().numpy(), ro) and np.array_equal(approx["ids"].cpu().numpy(), ri)
    e_ref = oracle.edges(data, lm, ro, ri, 4.0)
    assert np.array_equal(approx["edges"].cpu().numpy(), e_ref)
    exact_edges = set(map(tuple, exact["edges"].cpu().numpy().tolist()))
    assert set(map(tuple, e_ref.tolist())) <= exact_edges
    assert len(e_ref) < len(exact_edges)          # the index loses some edges at nprobe = 8


@pytest.mark.parametrize("path", ["tc", "fp32"])
def test_end_to_end_build(index, data, path):
    """End-to-end mode: the greedy driven by the index's range sets.  x is a landmark
    iff no earlier landmark's approximate ball holds x; the exact balls still cover X."""
    out = index.build(4.0, 4, path=path)
    lm = out["landmarks"].cpu().numpy()
    assert np.all(np.diff(lm) > 0)
    _, _, probes, _ = index.range_query(torch.from_numpy(data[lm]).cuda(), 4.0, 4)
    ro, ri = oracle.masked_range_query(data, data[lm], 4.0, index.cell_of.cpu().numpy(), 64, probes.cpu().numpy())
    assert np.array_equal(out["offsets"].cpu().numpy(), ro) and np.array_equal(out["ids"].cpu().numpy(), ri)
    n = data.shape[0]
    first_cover = np.full(n, n, dtype=np.int64)
    for k, l in enumerate(lm):
        members = ri[ro[k]:ro[k + 1]]
        first_cover[members] = np.minimum(first_cover[members], l)
    is_lm = np.zeros(n, bool)
    is_lm[lm] = True
    covered_earlier = first_cover < np.arange(n)
    assert np.array_equal(is_lm, ~covered_earlier)
    assert np.all(first_cover < n)                   # every point in some (exact) ball
    assert np.array_equal(out["edges"].cpu().numpy(), oracle.edges(data, lm, ro, ri, 4.0))


def test_tc_scan_on_ties_and_d128(bm):
    """The tensor-core scan on a tie-heavy grid (pairs at exactly eps, decided in the FP64
    recheck) and at d = 128 (the split's 256-wide point tiles), against the masked oracle."""
    G = W.tiny_grid_cloud(6000, 3, 2, span=8, seed=42)
    ig = bm.IvfIndex(torch.from_numpy(G).cuda(), nlist=16, iters=5, seed=1)
    for path in ("tc", "fp32"):
        off, ids, probes, _ = ig.range_query(torch.from_numpy(G[:500]).cuda(), 1.0, 3, path=path)
        ro, ri = oracle.masked_range_query(G, G[:500], 1.0, ig.cell_of.cpu().numpy(), 16, probes.cpu().numpy())
        assert np.array_equal(off.cpu().numpy(), ro) and np.array_equal(ids.cpu().numpy(), ri), path
    X = W.make("iso-n20k-d128")
    ix = bm.IvfIndex(torch.from_numpy(X).cuda(), nlist=32, iters=6, seed=2)
    off, ids, probes, _ = ix.range_query(torch.from_numpy(X[::23]).cuda(), 14.0, 5, path="tc")
    ro, ri = oracle.masked_range_query(X, X[::23], 14.0, ix.cell_of.cpu().numpy(), 32, probes.cpu().numpy())
    assert np.array_equal(off.cpu().numpy(), ro) and np.array_equal(ids.cpu().numpy(), ri)
