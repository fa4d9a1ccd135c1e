"""Batched builds (many independent instances, greedy loops inside one CUDA graph)
through the C-ABI, against the CPU oracle and against one bm_build per instance.

Every instance's landmarks, membership CSR and nerve edges must be bit-identical
to the oracle's for that instance alone: batching changes how the work is
scheduled on the device, never the result."""
import numpy as np
import pytest

import oracle
from paper_2601_01405_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PATHS = ["tc", "fp32", "tc16"]


@pytest.fixture(scope="module")
def bm():
    from paper_2601_01405_gb300 import _build, binding
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def to_np(out):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


def assert_same_graph(got, ref, tag=""):
    assert np.array_equal(got["landmarks"], ref["landmarks"]), ("landmarks", tag)
    assert np.array_equal(got["offsets"], ref["offsets"]), ("offsets", tag)
    assert np.array_equal(got["ids"], ref["ids"]), ("ids", tag)
    assert np.array_equal(got["edges"].reshape(-1, 2), ref["edges"].reshape(-1, 2)), ("edges", tag)


def mixed_instances():
    """Uneven sizes, dimensions and radii, with the degenerate cases: an empty
    instance, a single point, duplicates, a ball holding everything, and a
    coarse grid with many pairs at exactly eps."""
    out = []
    out.append((np.zeros((0, 5), dtype=np.float32), 1.0))
    out.append((np.ones((1, 3), dtype=np.float32), 0.5))
    out.append((np.full((40, 2), 0.25, dtype=np.float32), 1e-3))
    out.append((W.isotropic(3000, 8, 10, seed=1), 1.5))
    out.append((W.isotropic(700, 96, 10, seed=2), 12.0))
    out.append((W.mixture(5000, 32, 10, clusters=8, seed=3), 4.0))
    out.append((W.tiny_grid_cloud(4000, 3, 2, span=8, seed=4), 1.0))
    out.append((W.isotropic(129, 17, 10, seed=5), 1e3))
    out.append((W.isotropic(20000, 3, 10, seed=6), 0.3))
    out.append((W.swissroll(6000, 16, 12, seed=7), 0.8))
    return out


@pytest.mark.parametrize("path", PATHS)
def test_batched_matches_oracle(bm, path):
    inst = mixed_instances()
    res = bm.bm_build_batched([(torch.from_numpy(X).cuda(), e) for X, e in inst], path=path)
    torch.cuda.synchronize()
    assert len(res) == len(inst)
    for k, ((X, e), r) in enumerate(zip(inst, res)):
        ref = oracle.build(X, e)
        assert_same_graph(to_np(r), ref, (path, k))


@pytest.mark.parametrize("path", PATHS)
def test_batched_equals_single_builds(bm, path):
    """A slice of the batched workload recipe (n log-uniform, d in {8, 32, 96},
    isotropic or 8 clusters, own eps in [1, 5]) at reduced n: batched == bm_build."""
    inst = W.batched_instances(count=24, seed=11, n_hi=30000)
    dev = [(torch.from_numpy(i.x).cuda(), i.eps) for i in inst]
    res = bm.bm_build_batched(dev, path=path)
    for k, ((Xd, e), r) in enumerate(zip(dev, res)):
        single = bm.bm_build(Xd, e, path=path)
        torch.cuda.synchronize()
        assert_same_graph(to_np(r), to_np(single), (path, k))
        assert r["stats"]["kernel_launches"] > 0


def test_batched_host_io(bm):
    inst = mixed_instances()[:6]
    host = bm.bm_build_batched(inst)
    dev = bm.bm_build_batched([(torch.from_numpy(X).cuda(), e) for X, e in inst])
    for k, (h, d_) in enumerate(zip(host, dev)):
        assert isinstance(h["ids"], np.ndarray)
        assert_same_graph(h, to_np(d_), k)


def test_batched_small_batch_option(bm):
    """The largest candidate batch per step is an option; results do not depend on it."""
    inst = [(W.isotropic(5000, 8, 10, seed=31), 1.2), (W.mixture(8000, 32, 10, clusters=8, seed=32), 3.0)]
    dev = [(torch.from_numpy(X).cuda(), e) for X, e in inst]
    a = bm.bm_build_batched(dev, batch=64)
    b = bm.bm_build_batched(dev, batch=2048)
    for k, (x, y) in enumerate(zip(a, b)):
        assert_same_graph(to_np(x), to_np(y), k)
        assert_same_graph(to_np(x), oracle.build(*inst[k]), k)


def test_batched_rejects_nan_instance(bm):
    good = torch.from_numpy(W.isotropic(500, 4, 10, seed=41)).cuda()
    bad = good.clone()
    bad[7, 1] = float("nan")
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_build_batched([(good, 1.0), (bad, 1.0), (good, 2.0)])
    assert ei.value.status == bm.BM_ERR_ARG
    assert "instance 1" in str(ei.value)
    # the library stays usable
    r = bm.bm_build_batched([(good, 1.0)])
    assert_same_graph(to_np(r[0]), oracle.build(good.cpu().numpy(), 1.0))


def test_batched_empty_list(bm):
    assert bm.bm_build_batched([]) == []


def test_batched_auto_picks_a_path_per_instance(bm):
    """The automatic path's first step runs every instance on the split and moves the
    well-separated ones to fp16 before the graph; a Swiss roll (wide fp16 band) stays on
    the split.  Every result equals the oracle's."""
    inst = [(W.mixture(6000, 64, 8, clusters=8, seed=51), 2.0),
            (W.swissroll(8000, 128, 12, seed=52), 0.5),
            (W.isotropic(3000, 32, 10, seed=53), 1.0)]
    res = bm.bm_build_batched([(torch.from_numpy(X).cuda(), e) for X, e in inst])
    torch.cuda.synchronize()
    paths = [r["stats"]["path"] for r in res]
    assert paths[0] == bm.BM_PATH_TC_FP16
    assert paths[1] == bm.BM_PATH_TC_SPLIT3
    for k, ((X, e), r) in enumerate(zip(inst, res)):
        assert_same_graph(to_np(r), oracle.build(X, e), k)


def test_batched_per_instance_batches(bm):
    """Per-instance largest batches (what the autotuned table supplies) change the schedule,
    never the result."""
    from paper_2601_01405_gb300 import autotune
    inst = W.batched_instances(count=9, seed=61, n_hi=20000)
    dev = [(torch.from_numpy(i.x).cuda(), i.eps) for i in inst]
    table = {8: [{"n_lo": 1000, "n_hi": 5000, "best": 128}, {"n_lo": 5000, "n_hi": 200000, "best": 2048}],
             32: [{"n_lo": 1000, "n_hi": 200000, "best": 256}], 96: [{"n_lo": 1000, "n_hi": 200000, "best": 512}]}
    per = autotune.batches_for(table, dev)
    assert set(per) <= {128, 256, 512, 2048}
    a = bm.bm_build_batched(dev, batches=per)
    b = bm.bm_build_batched(dev)
    for k, (x, y) in enumerate(zip(a, b)):
        assert_same_graph(to_np(x), to_np(y), k)
    with pytest.raises(bm.BallMapperError):
        bm.bm_build_batched(dev, batches=[48] * len(dev))
