"""Nerve edges (Sec. 5.2) through both deduplications -- the landmark-row bitmap
(one chunk, and many small chunks) and the sort of pair keys -- against the CPU
oracle, in single and batched builds."""
import numpy as np
import pytest

import oracle
from paper_2601_01405_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# bitmap budgets: default (one chunk here), always sort, a few rows per chunk
BUDGETS = [0, -1, 4096]


@pytest.fixture(scope="module")
def bm():
    from paper_2601_01405_gb300 import _build, binding
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield binding
    binding.set_nerve_bitmap_bytes(0)


def cases():
    return [(W.isotropic(5000, 8, 10, seed=1), 2.0),                 # dense witnesses
            (W.tiny_grid_cloud(3000, 3, 2, span=8, seed=2), 1.25),    # ties at eps
            (W.mixture(8000, 16, 10, clusters=8, seed=3), 5.0),       # many overlapping balls
            (W.isotropic(20000, 32, 10, seed=4), 5.0),                # sparse witnesses, L close to n
            (W.swissroll(30000, 24, 12, seed=5), 0.6)]


@pytest.mark.parametrize("budget", BUDGETS)
def test_nerve_paths_match_oracle(bm, budget):
    bm.set_nerve_bitmap_bytes(budget)
    try:
        for k, (X, eps) in enumerate(cases()):
            out = bm.bm_build(torch.from_numpy(X).cuda(), eps)
            torch.cuda.synchronize()
            ref = oracle.build(X, eps)
            assert np.array_equal(out["landmarks"].cpu().numpy(), ref["landmarks"]), (budget, k)
            got = out["edges"].cpu().numpy().reshape(-1, 2)
            assert np.array_equal(got, ref["edges"].reshape(-1, 2)), (budget, k, got.shape, ref["edges"].shape)
            assert out["stats"]["edge_pairs"] >= got.shape[0]
    finally:
        bm.set_nerve_bitmap_bytes(0)


@pytest.mark.parametrize("budget", BUDGETS)
def test_nerve_paths_batched(bm, budget):
    cs = cases()
    bm.set_nerve_bitmap_bytes(budget)
    try:
        res = bm.bm_build_batched([(torch.from_numpy(X).cuda(), e) for X, e in cs])
        torch.cuda.synchronize()
        for k, ((X, eps), r) in enumerate(zip(cs, res)):
            ref = oracle.build(X, eps)
            assert np.array_equal(r["edges"].cpu().numpy().reshape(-1, 2), ref["edges"].reshape(-1, 2)), (budget, k)
            assert np.array_equal(r["ids"].cpu().numpy(), ref["ids"]), (budget, k)
    finally:
        bm.set_nerve_bitmap_bytes(0)
