"""k-th nearest-neighbour distances and the target-occupancy scale (Sec. 6.1) on the
GPU, through the C-ABI, against the CPU oracle.

kdist[i] is sqrt of the k-th smallest FP64 squared distance from point i to all
points, itself included; the GPU takes the same FP64 value (its select works on the
oracle's arithmetic), so the comparison is exact, element by element.  The
occupancy eps is the median of kdist, and the paper's worked example (Sec. 6.3) is
run end to end on the float32 cast of its Gaussian."""
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


def knn(bm, X, k, path="auto"):
    kd, st = bm.bm_knn_dist(torch.from_numpy(np.ascontiguousarray(X)).cuda(), k, path=path)
    torch.cuda.synchronize()
    return kd.cpu().numpy(), st


@pytest.mark.parametrize("path", ["auto", "tc", "fp32"])
@pytest.mark.parametrize("k", [1, 2, 50])
def test_knn_iso_n10k_d16(bm, path, k):
    X = W.make("iso-n10k-d16")
    got, st = knn(bm, X, k, path)
    assert np.array_equal(got, oracle.kth_nn_dist(X, k))
    if k == 1:
        assert np.all(got == 0.0)          # itself, counted first


@pytest.mark.parametrize("k", [7, 37, 300])
def test_knn_ties_and_duplicates(bm, k):
    """Integer-grid cloud: many equal distances and duplicate points."""
    X = W.tiny_grid_cloud(5000, 3, 2, span=6, seed=51)
    got, _ = knn(bm, X, k)
    assert np.array_equal(got, oracle.kth_nn_dist(X, k))


@pytest.mark.parametrize("name,k", [("mix32-n32k-d64", 50), ("roll-n50k-d128", 20), ("iso-n20k-d128", 50)])
def test_knn_reduced_workloads(bm, name, k):
    X = W.make(name)
    got, st = knn(bm, X, k)
    ref = oracle.kth_nn_dist(X, k)
    assert np.array_equal(got, ref)
    assert st["tile_pairs"] == X.shape[0] ** 2


def test_knn_edge_cases(bm):
    X = np.full((300, 5), 0.75, dtype=np.float32)      # all identical
    got, _ = knn(bm, X, 300)
    assert np.all(got == 0.0)
    Y = W.isotropic(5, 3, 10, seed=52)                  # k = n, tiny n
    got, _ = knn(bm, Y, 5)
    assert np.array_equal(got, oracle.kth_nn_dist(Y, 5))
    Z = W.isotropic(1, 4, 10, seed=53)                  # a single point
    got, _ = knn(bm, Z, 1)
    assert got.tolist() == [0.0]
    U = (W.isotropic(4000, 33, 10, seed=54).astype(np.float64) * 1e6 + 3e7).astype(np.float32)  # wide band
    got, _ = knn(bm, U, 25)
    assert np.array_equal(got, oracle.kth_nn_dist(U, 25))


def test_knn_host_io_and_errors(bm):
    X = W.isotropic(3000, 9, 10, seed=55)
    kd, _ = bm.bm_knn_dist(X, 12)
    assert isinstance(kd, np.ndarray) and np.array_equal(kd, oracle.kth_nn_dist(X, 12))
    Xd = torch.from_numpy(X).cuda()
    for bad_k in (0, 3001, 1025):
        with pytest.raises(bm.BallMapperError) as ei:
            bm.bm_knn_dist(Xd, bad_k)
        assert ei.value.status == bm.BM_ERR_ARG
    Xn = Xd.clone()
    Xn[100, 3] = float("nan")
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_knn_dist(Xn, 5)
    assert ei.value.status == bm.BM_ERR_ARG


@pytest.mark.parametrize("n", [9999, 10000])
def test_occupancy_eps_matches_oracle(bm, n):
    """Odd and even counts (the even median is the mean of the two middle values)."""
    X = W.make("iso-n10k-d16")[:n]
    eps, _ = bm.bm_occupancy_eps(torch.from_numpy(X).cuda(), 20)
    assert eps == oracle.occupancy_eps(X, 20)


def test_paper_worked_example_end_to_end(bm):
    """Sec. 6.3: Gaussian n = 20000, d = 50, k = 50 (printed: eps ~ 7.5536, 6361
    landmarks, 936,690 edges, from FP64 data).  The GPU takes float32 coordinates, so
    the data is the float32 cast of the same draws; eps and the whole Ball Mapper must
    equal the oracle's on those same bytes, and the counts equal the printed ones."""
    X = W.paper_gaussian_fp64(20000, 50, seed=0).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    eps, st = bm.bm_occupancy_eps(Xd, 50)
    ref_eps = oracle.occupancy_eps(X, 50)
    assert eps == ref_eps
    assert abs(eps - 7.5536) < 1e-3
    e32 = float(np.float32(eps))
    out = bm.bm_build(Xd, e32)
    torch.cuda.synchronize()
    ref = oracle.build(X, e32)
    assert np.array_equal(out["landmarks"].cpu().numpy(), ref["landmarks"])
    assert np.array_equal(out["ids"].cpu().numpy(), ref["ids"])
    assert np.array_equal(out["edges"].cpu().numpy(), ref["edges"])
    # the float32 cast keeps the printed counts
    assert ref["landmarks"].size == 6361 and ref["edges"].shape[0] == 936690
