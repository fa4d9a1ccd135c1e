"""bm_range_count_noalloc, the entry point that allocates nothing.

It serves callers that cannot allocate device memory when they call
(allocation-free real-time code, code inside another allocator's callback,
fixed memory budgets): it works in scratch compiled into the library.  Here it
is called through the C-ABI and its counts are checked, element by element,
against the CPU oracle's range sets and against the row lengths of the regular
range-query entry point, on two calls in a row with different shapes (so that
anything the first call leaves in the shared scratch would show).  Its error
paths are covered too: NaN input, more boundary pairs than the scratch holds,
and an eps beyond its limit."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bm():
    from paper_2601_01405_gb300 import _build, binding
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def _check(bm, X, Q, eps):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    counts = torch.full((Q.shape[0],), -7, dtype=torch.int64, device="cuda")
    bm.bm_range_count_noalloc(Xd, Qd, eps, counts)
    off, ids, _ = bm.bm_range_query(Xd, Qd, eps, path="tc")
    torch.cuda.synchronize()
    got = counts.cpu().numpy()
    ref_off, _ = oracle.range_query(X, Q, eps)
    assert np.array_equal(got, np.diff(ref_off))          # the oracle's exact range sets
    assert np.array_equal(got, np.diff(off.cpu().numpy()))  # the allocating entry point
    return got


def test_noalloc_counts_match_oracle_on_two_calls(bm):
    from paper_2601_01405_gb300 import workloads as W
    X1 = W.isotropic(20000, 16, 10, seed=31)
    c1 = _check(bm, X1, X1[:777], 3.0)
    assert int(c1.min()) >= 1                      # every query is a point of X: its own ball holds it
    X2 = W.tiny_grid_cloud(8000, 3, 2, span=8, seed=32)   # many pairs at exactly eps: band recheck
    c2 = _check(bm, X2, X2[:900], 1.0)
    assert int(c2.sum()) > 900


def test_noalloc_queries_not_in_the_point_set(bm):
    from paper_2601_01405_gb300 import workloads as W
    X = W.mixture(12000, 24, 8, clusters=6, seed=33)
    Q = W.isotropic(301, 24, 8, seed=34) * np.float32(4.0)
    _check(bm, X, Q, 6.0)


def test_noalloc_rejects_nan(bm):
    X = torch.zeros((100, 3), dtype=torch.float32, device="cuda")
    X[17, 2] = float("nan")
    Q = torch.zeros((5, 3), dtype=torch.float32, device="cuda")
    counts = torch.zeros(5, dtype=torch.int64, device="cuda")
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_range_count_noalloc(X, Q, 1.0, counts)
    assert ei.value.status == bm.BM_ERR_ARG
    # the next call on clean data is unaffected by the flag the failed call left in the scratch
    X[17, 2] = 0.0
    bm.bm_range_count_noalloc(X, Q, 1.0, counts)
    torch.cuda.synchronize()
    assert counts.cpu().tolist() == [100] * 5


def test_noalloc_band_overflow_is_reported(bm):
    """2100 x 1000 pairs at squared distance exactly eps^2: all of them lie in the error
    band, more than the 2,097,120 band slots of the scratch."""
    X = torch.zeros((2100, 1), dtype=torch.float32, device="cuda")
    Q = torch.full((1000, 1), 0.5, dtype=torch.float32, device="cuda")
    counts = torch.zeros(1000, dtype=torch.int64, device="cuda")
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_range_count_noalloc(X, Q, 0.5, counts)
    assert ei.value.status == bm.BM_ERR_CAPACITY


def test_noalloc_rejects_sizes_beyond_its_scratch(bm):
    X = torch.zeros((4_194_304, 1), dtype=torch.float32, device="cuda")
    Q = torch.zeros((1, 1), dtype=torch.float32, device="cuda")
    counts = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_range_count_noalloc(X, Q, 1.0, counts)
    assert ei.value.status == bm.BM_ERR_CAPACITY
    assert "scratch" in str(ei.value)
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_range_count_noalloc(Q, Q, 1e20, counts)
    assert ei.value.status == bm.BM_ERR_ARG
