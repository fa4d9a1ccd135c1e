"""Every compiled tensor-core tile shape, at every padding the library accepts,
gives results identical to the CPU oracle (range sets) and to the built-in
configuration (whole builds): the tile configuration changes speed only."""
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
def autotune(bm):
    from paper_2601_01405_gb300 import autotune
    return autotune


@pytest.mark.parametrize("d,eps", [(8, 1.5), (33, 5.0), (96, 11.0), (128, 13.0)])
def test_every_tile_config_matches_oracle(bm, autotune, d, eps):
    X = W.isotropic(3000, d, 10, seed=d)
    Q = W.isotropic(300, d, 10, seed=d + 1)
    ro, ri = oracle.range_query(X, Q, eps)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    cfgs = autotune.candidates(d)
    assert len(cfgs) >= 2
    try:
        for cfg in cfgs:
            bm.set_tile_config(d, cfg)
            off, ids, _ = bm.bm_range_query(Xd, Qd, eps)
            torch.cuda.synchronize()
            assert np.array_equal(off.cpu().numpy(), ro), cfg
            assert np.array_equal(ids.cpu().numpy(), ri), cfg
    finally:
        bm.set_tile_config(d, None)


def test_build_under_each_config_equals_builtin(bm, autotune):
    X = W.mixture(20000, 96, 10, clusters=8, seed=5)
    Xd = torch.from_numpy(X).cuda()
    ref = bm.bm_build(Xd, 9.0)
    torch.cuda.synchronize()
    try:
        for cfg in autotune.candidates(96):
            bm.set_tile_config(96, cfg)
            out = bm.bm_build(Xd, 9.0)
            torch.cuda.synchronize()
            for k in ("landmarks", "offsets", "ids", "edges"):
                assert torch.equal(out[k], ref[k]), (cfg, k)
    finally:
        bm.set_tile_config(96, None)
