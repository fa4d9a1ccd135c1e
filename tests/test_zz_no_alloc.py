"""bm_range_count_noalloc, the entry point that allocates nothing.

It serves callers that cannot allocate device memory when they call (inside a
stream capture, allocation-free real-time code, fixed memory budgets): it
works in scratch compiled into the library.  Here it is called through the
C-ABI and its counts are checked against the row lengths returned by the
regular range-query entry point, on two calls in a row with different shapes
(so that anything the first call leaves in the shared scratch would show)."""
import numpy as np
import pytest

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
    assert torch.equal(counts, off[1:] - off[:-1])
    return counts


def test_noalloc_counts_match_range_query_on_two_calls(bm):
    from paper_2601_01405_gb300 import workloads as W
    X1 = W.isotropic(20000, 16, 10, seed=31)
    c1 = _check(bm, X1, X1[:777], 3.0)
    assert int(c1.min()) >= 1                      # every query is a point of X: its own ball holds it
    X2 = W.tiny_grid_cloud(8000, 3, 2, span=8, seed=32)   # many pairs at exactly eps: band recheck
    c2 = _check(bm, X2, X2[:900], 1.0)
    assert int(c2.sum()) > 900


def test_noalloc_rejects_sizes_beyond_its_scratch(bm):
    X = torch.zeros((4_194_304, 1), dtype=torch.float32, device="cuda")
    Q = torch.zeros((1, 1), dtype=torch.float32, device="cuda")
    counts = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_range_count_noalloc(X, Q, 1.0, counts)
    assert ei.value.status == bm.BM_ERR_CAPACITY
    assert "scratch" in str(ei.value)
