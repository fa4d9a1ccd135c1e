"""Translated tensor-core operands (bm_options.centring) against the CPU oracle.

D(q, x) does not change when points and queries move by the same vector, so every
landmark, membership and edge must equal the oracle's whether or not the tiles work on
x - c; only the proven band (which grows with the operands' norms) may change."""
import numpy as np
import pytest

import oracle
from paper_2601_01405_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OFFSET = 12.0


@pytest.fixture(scope="module")
def bm():
    from paper_2601_01405_gb300 import _build, binding
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def cuda(X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()


def to_np(out):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


def run_build(bm, X, eps, path, centring):
    out = bm.bm_build(cuda(X), eps, path=path, centring=centring)
    torch.cuda.synchronize()
    return to_np(out)


def assert_same_graph(got, ref, tag=""):
    assert np.array_equal(got["landmarks"], ref["landmarks"]), ("landmarks", tag)
    assert np.array_equal(got["offsets"], ref["offsets"]), ("offsets", tag)
    assert np.array_equal(got["ids"], ref["ids"]), ("ids", tag)
    assert np.array_equal(got["edges"].reshape(-1, 2), ref["edges"].reshape(-1, 2)), ("edges", tag)


def shifted(n, d, seed, offset=OFFSET):
    """Isotropic cloud moved away from the origin: multiples of 2^-10 below 2^5, exact
    in float32, so the oracle's FP64 distances are exact."""
    return (W.isotropic(n, d, 10, seed=seed).astype(np.float64) + offset).astype(np.float32)


@pytest.mark.parametrize("path", ["tc", "tc16", "auto"])
@pytest.mark.parametrize("centring", ["always", "off", "auto"])
def test_translated_build_matches_oracle(bm, path, centring):
    X = shifted(4000, 16, seed=1)
    got = run_build(bm, X, 3.0, path, centring)
    assert_same_graph(got, oracle.build(X, 3.0), (path, centring))
    # automatic mode translates only from 65,536 points on
    assert got["stats"]["centred"] == (1 if centring == "always" else 0)


def test_translation_shrinks_the_band(bm):
    """Norms ~50 against a spread of ~4: the translated band is far narrower and far
    fewer pairs need the FP64 recheck; the graph is the same."""
    X = shifted(3000, 16, seed=2)
    on = run_build(bm, X, 3.0, "tc", "always")
    off = run_build(bm, X, 3.0, "tc", "off")
    assert_same_graph(on, off)
    assert on["stats"]["band_delta"] * 10 < off["stats"]["band_delta"]
    assert on["stats"]["band_pairs"] < off["stats"]["band_pairs"]


@pytest.mark.parametrize("centring", ["always", "off"])
@pytest.mark.parametrize("path", ["tc", "tc16"])
def test_translated_range_query_with_far_queries(bm, centring, path):
    """The queries move with the points' centre: queries on the points, far on the other
    side of the origin, and next to the cloud."""
    X = shifted(5000, 24, seed=3)
    Q = np.concatenate([X[::11], shifted(200, 24, seed=4, offset=-20.0), shifted(100, 24, seed=5, offset=12.5)])
    off, ids, st = bm.bm_range_query(cuda(X), cuda(Q), 3.5, path=path, centring=centring)
    torch.cuda.synchronize()
    ro, ri = oracle.range_query(X, Q, 3.5)
    assert np.array_equal(off.cpu().numpy(), ro)
    assert np.array_equal(ids.cpu().numpy(), ri)
    assert st["centred"] == (1 if centring == "always" else 0)


def test_translated_range_query_with_distances(bm):
    X = shifted(3000, 12, seed=12, offset=-9.0)
    Q = X[::5]
    off, ids, st, dists = bm.bm_range_query(cuda(X), cuda(Q), 2.5, path="tc", centring="always", want_dists=True)
    torch.cuda.synchronize()
    ro, ri = oracle.range_query(X, Q, 2.5)
    assert np.array_equal(off.cpu().numpy(), ro) and np.array_equal(ids.cpu().numpy(), ri)
    rows = np.repeat(np.arange(Q.shape[0]), np.diff(ro))
    ref = np.sqrt(((Q[rows].astype(np.float64) - X[ri].astype(np.float64)) ** 2).sum(-1))
    got = dists.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-6 * np.maximum(ref, 1e-30))
    assert st["centred"] == 1


def test_auto_translates_large_off_centre_sets(bm):
    """Swiss roll (mean far from the origin, 70,000 points): the automatic mode
    translates, and the build equals the oracle."""
    X = W.swissroll(70_000, 16, 12, seed=6)
    got = run_build(bm, X, 1.5, "auto", "auto")
    assert got["stats"]["centred"] == 1
    assert_same_graph(got, oracle.build(X, 1.5))


def test_auto_leaves_centred_sets_alone(bm):
    """An isotropic cloud around the origin: translating by its sample mean cannot
    shrink the largest norm by 5 %, so the automatic mode keeps the coordinates."""
    X = W.isotropic(70_000, 8, 10, seed=7)
    got = run_build(bm, X, 2.5, "auto", "auto")
    assert got["stats"]["centred"] == 0
    ref = run_build(bm, X, 2.5, "auto", "off")
    assert_same_graph(got, ref)


def test_forced_translation_that_widens_the_band(bm):
    """Most points near e1 and one far point at -3 e1: the mean sits near e1, so the
    translated norms grow (the far point moves to ~4).  Forced translation must stay
    exact; the automatic decision (at this size it does not apply) is not involved."""
    rng = np.random.default_rng(8)
    X = 0.05 * rng.standard_normal((3000, 6))
    X[:, 0] += 1.0
    X[-1] = 0.0
    X[-1, 0] = -3.0
    X = W.quantise(X, 10)
    for path in ("tc", "tc16"):
        got = run_build(bm, X, 0.1, path, "always")
        assert got["stats"]["centred"] == 1
        assert_same_graph(got, oracle.build(X, 0.1), path)


def test_batched_translation(bm):
    inst = [(shifted(3000, 8, seed=9), 2.0), (W.isotropic(2000, 32, 10, seed=10), 6.0),
            (shifted(1500, 96, seed=11, offset=-6.0), 12.0)]
    res = bm.bm_build_batched([(cuda(X), e) for X, e in inst], centring="always")
    torch.cuda.synchronize()
    for k, ((X, e), r) in enumerate(zip(inst, res)):
        assert_same_graph(to_np(r), oracle.build(X, e), k)
        assert r["stats"]["centred"] == 1


@pytest.mark.parametrize("centring", ["always", "off"])
def test_translated_knn_matches_oracle(bm, centring):
    """The k-NN sweep (each row with its own squared radius) on translated operands."""
    X = shifted(6000, 12, seed=13)
    kd, st = bm.bm_knn_dist(cuda(X), 6, centring=centring)
    torch.cuda.synchronize()
    assert np.array_equal(kd.cpu().numpy(), oracle.kth_nn_dist(X, 6))
    assert st["centred"] == (1 if centring == "always" else 0)


def test_auto_translation_on_large_knn(bm):
    """70,000 points far from the origin: the automatic mode translates the k-NN sweep."""
    X = shifted(70_000, 8, seed=51, offset=9.0)
    kd, st = bm.bm_knn_dist(cuda(X), 6)
    torch.cuda.synchronize()
    assert st["centred"] == 1
    assert np.array_equal(kd.cpu().numpy(), oracle.kth_nn_dist(X, 6))
