"""CUDA path (through the C-ABI) against the CPU oracle, element by element.

Landmarks, membership CSR and nerve edges are integer / index results and must
be bit-identical to the oracle on the same seeded inputs, on every distance-tile
path (bf16 split and fp16 tensor-core tiles, FP32 CUDA-core tiles)."""
import numpy as np
import pytest

import oracle
from paper_2601_01405_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PATHS = ["tc", "fp32", "tc16", "auto"]


@pytest.fixture(scope="module")
def bm():
    from paper_2601_01405_gb300 import _build, binding
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def run_build(bm, X, eps, path, batch=0):
    out = bm.bm_build(torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda(), eps, path=path, batch=batch)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


def assert_same_graph(got, ref, tag=""):
    assert np.array_equal(got["landmarks"], ref["landmarks"]), ("landmarks", tag)
    assert np.array_equal(got["offsets"], ref["offsets"]), ("offsets", tag)
    assert np.array_equal(got["ids"], ref["ids"]), ("ids", tag)
    assert np.array_equal(got["edges"].reshape(-1, 2), ref["edges"].reshape(-1, 2)), ("edges", tag)


# ------------------------------------------------------------------ range query
@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n,m,d,eps", [(10_000, 777, 16, 3.0), (4099, 300, 3, 0.4), (5000, 129, 17, 2.5),
                                       (3000, 1000, 64, 9.5), (2500, 257, 100, 12.0), (1, 5, 8, 1.0),
                                       (700, 1, 128, 14.0), (1000, 64, 1, 0.01)])
def test_range_query_matches_oracle(bm, path, n, m, d, eps):
    X = W.isotropic(n, d, 10, seed=n + d)
    Q = W.isotropic(m, d, 10, seed=m + 3 * d)
    off, ids, st = bm.bm_range_query(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), eps, path=path)
    torch.cuda.synchronize()
    ro, ri = oracle.range_query(X, Q, eps)
    assert np.array_equal(off.cpu().numpy(), ro)
    assert np.array_equal(ids.cpu().numpy(), ri)
    assert st["distance_evals"] == n * m


@pytest.mark.parametrize("path", PATHS)
def test_range_query_ties_on_grid(bm, path):
    """Coarse grid data: many pairs at exactly eps; open balls exclude them."""
    X = W.tiny_grid_cloud(6000, 3, 2, span=8, seed=1)
    for eps in (0.5, 1.0, 1.25):
        off, ids, st = bm.bm_range_query(torch.from_numpy(X).cuda(), torch.from_numpy(X[:900]).cuda(), eps, path=path)
        ro, ri = oracle.range_query(X, X[:900], eps)
        assert np.array_equal(off.cpu().numpy(), ro) and np.array_equal(ids.cpu().numpy(), ri), eps
        assert st["band_pairs"] > 0   # the exact ties must have gone through the FP64 recheck


@pytest.mark.parametrize("path", PATHS)
def test_range_query_host_io(bm, path):
    X = W.isotropic(3000, 32, 10, seed=5)
    Q = X[::7]
    off, ids, _ = bm.bm_range_query(X, Q, 4.0, path=path)
    ro, ri = oracle.range_query(X, Q, 4.0)
    assert isinstance(off, np.ndarray)
    assert np.array_equal(off, ro) and np.array_equal(ids, ri)


@pytest.mark.parametrize("path", PATHS)
def test_range_query_empty(bm, path):
    X = W.isotropic(100, 4, 10, seed=1)
    off, ids, _ = bm.bm_range_query(torch.from_numpy(X).cuda(), torch.zeros((0, 4)).cuda(), 1.0, path=path)
    assert off.cpu().tolist() == [0] and ids.numel() == 0
    off, ids, _ = bm.bm_range_query(torch.zeros((0, 4)).cuda(), torch.from_numpy(X[:5]).cuda(), 1.0, path=path)
    assert off.cpu().tolist() == [0] * 6 and ids.numel() == 0


# ------------------------------------------------------------------ build
@pytest.mark.parametrize("path", PATHS)
def test_build_golden_line_and_grid(bm, path):
    import pins
    for case in pins.golden("line.json")["cases"]:
        got = run_build(bm, W.line_points(10, 3), case["eps"], path)
        assert got["landmarks"].tolist() == case["landmarks"]
        assert pins.rows(got["offsets"], got["ids"]) == case["members"]
        assert got["edges"].tolist() == case["edges"]
    for case in pins.golden("grid.json")["cases"]:
        got = run_build(bm, W.grid_points(3), case["eps"], path)
        assert got["landmarks"].tolist() == case["landmarks"]
        assert pins.rows(got["offsets"], got["ids"]) == case["members"]
        assert got["edges"].tolist() == case["edges"]


@pytest.mark.parametrize("path", PATHS)
def test_build_iso_n10k_d16(bm, path):
    X = W.make("iso-n10k-d16")
    ref = oracle.build(X, 3.0)
    got = run_build(bm, X, 3.0, path)
    assert_same_graph(got, ref)
    assert got["stats"]["distance_evals"] == ref["landmarks"].size * X.shape[0]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("batch", [32, 96, 1024, 2048, 4096, 8192, 16384])
def test_build_batch_sizes(bm, path, batch):
    X = W.isotropic(5003, 8, 10, seed=3)
    ref = oracle.build(X, 2.0)
    assert_same_graph(run_build(bm, X, 2.0, path, batch=batch), ref, batch)


@pytest.mark.parametrize("path", PATHS)
def test_build_batch_8192_conflicts(bm, path):
    """Isolated points (a 2000-wide cube in 6-d, eps 1) with near copies planted
    every 131st index, each within 8,000 positions of its original: over 99 % of
    the candidates survive, the batch grows to 8192 (steps of 256, 512, ..., 8192,
    8192, 8192), and the in-batch conflicts fall in every word of the candidate set
    (the last killed slot is 8176)."""
    rng = np.random.default_rng(5)
    n = 26000
    X = np.round(rng.uniform(-1000.0, 1000.0, (n, 6)) * 16.0) / 16.0
    for i in range(40, n, 131):
        j = i - int(rng.integers(1, min(i, 8000) + 1))
        X[i] = X[j] + rng.integers(-4, 5, 6) / 16.0   # within sqrt(6)/4 < 1 of X[j]
    X = X.astype(np.float32)
    ref = oracle.build(X, 1.0)
    assert n - ref["landmarks"].size == 199
    got = run_build(bm, X, 1.0, path, batch=8192)
    assert_same_graph(got, ref)
    assert got["stats"]["greedy_steps"] < 10   # 8 steps; a batch capped at 4096 takes 10


@pytest.mark.parametrize("path", ["tc", "auto"])
def test_build_batch_16384_conflicts(bm, path):
    """The largest batch of a single build: isolated points with near copies planted
    every 97th index, each within 16,000 positions of its original, so the batch grows to
    16384 (the default) and in-batch conflicts fall across all 512 words of a conflict row."""
    rng = np.random.default_rng(6)
    n = 60000
    X = np.round(rng.uniform(-1000.0, 1000.0, (n, 6)) * 16.0) / 16.0
    for i in range(40, n, 97):
        j = i - int(rng.integers(1, min(i, 16000) + 1))
        X[i] = X[j] + rng.integers(-4, 5, 6) / 16.0   # within sqrt(6)/4 < 1 of X[j]
    X = X.astype(np.float32)
    ref = oracle.build(X, 1.0)
    assert n - ref["landmarks"].size > 500
    got = run_build(bm, X, 1.0, path)
    assert_same_graph(got, ref)
    assert got["stats"]["greedy_steps"] < 11   # 256, 512, ..., 16384, 16384, rest: 9 steps; capped at 8192: 12


@pytest.mark.parametrize("path", PATHS)
def test_build_mixture_d64(bm, path):
    X = W.mixture(8192, 64, 8, clusters=32, seed=0)
    for eps in (6.0, 11.0, 12.5):
        ref = oracle.build(X, eps)
        assert_same_graph(run_build(bm, X, eps, path), ref, eps)


@pytest.mark.parametrize("path", PATHS)
def test_build_swissroll_d128(bm, path):
    X = W.swissroll(12000, 128, 12, seed=0)
    for eps in (1.0, 2.0):
        ref = oracle.build(X, eps)
        assert_same_graph(run_build(bm, X, eps, path), ref, eps)


@pytest.mark.parametrize("path", PATHS)
def test_build_degenerate(bm, path):
    # n = 0
    got = run_build(bm, np.zeros((0, 3), np.float32), 1.0, path)
    assert got["landmarks"].size == 0 and got["offsets"].tolist() == [0] and got["edges"].size == 0
    # n = 1
    got = run_build(bm, np.ones((1, 5), np.float32), 0.5, path)
    assert got["landmarks"].tolist() == [0] and got["ids"].tolist() == [0]
    # identical points
    got = run_build(bm, np.full((300, 2), 0.5, np.float32), 1e-3, path)
    assert got["landmarks"].tolist() == [0] and got["ids"].tolist() == list(range(300))
    # eps larger than the diameter
    X = W.isotropic(2000, 6, 10, seed=2)
    got = run_build(bm, X, 1e4, path)
    assert got["landmarks"].tolist() == [0] and got["ids"].tolist() == list(range(2000))
    # d = 1
    X = W.isotropic(3000, 1, 10, seed=9)
    assert_same_graph(run_build(bm, X, 0.05, path), oracle.build(X, 0.05))


@pytest.mark.parametrize("path", PATHS)
def test_build_grid_ties(bm, path):
    X = W.tiny_grid_cloud(4000, 3, 2, span=8, seed=4)
    for eps in (0.5, 1.0, 1.5):
        assert_same_graph(run_build(bm, X, eps, path), oracle.build(X, eps), eps)


@pytest.mark.parametrize("path", PATHS)
def test_build_unquantised_fp32(bm, path):
    """Arbitrary float32 input: the FP64 recheck reproduces the oracle's arithmetic."""
    X = np.random.default_rng(5).standard_normal((6000, 20)).astype(np.float32)
    assert_same_graph(run_build(bm, X, 4.0, path), oracle.build(X, 4.0))


@pytest.mark.parametrize("path", PATHS)
def test_build_host_io_and_determinism(bm, path):
    X = W.isotropic(4000, 16, 10, seed=11)
    a = bm.bm_build(X, 3.0, path=path)
    b = run_build(bm, X, 3.0, path)
    c = run_build(bm, X, 3.0, path)
    for k in ("landmarks", "offsets", "ids", "edges"):
        assert np.array_equal(a[k], b[k]) and np.array_equal(b[k], c[k]), k


def test_paths_agree_on_paper_gaussian_fp32(bm):
    """The paper's worked example (Sec. 6.3) cast to float32: all paths agree with
    each other and with the oracle on the same float32 data."""
    X = W.paper_gaussian_fp64().astype(np.float32)
    eps = float(np.float32(7.553576))
    ref = oracle.build(X, eps)
    for path in PATHS:
        assert_same_graph(run_build(bm, X, eps, path), ref, path)


# ------------------------------------------------------------------ errors
def test_errors_are_reported(bm):
    X = torch.from_numpy(W.isotropic(100, 4, 10, seed=1)).cuda()
    for bad_eps in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(bm.BallMapperError) as ei:
            bm.bm_build(X, bad_eps)
        assert ei.value.status == bm.BM_ERR_ARG
    Xn = X.clone()
    Xn[3, 1] = float("nan")
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_build(Xn, 1.0)
    assert ei.value.status == bm.BM_ERR_ARG
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_build(X, 1.0, batch=33)
    assert ei.value.status == bm.BM_ERR_ARG


# ------------------------------------------------------------------ buffer growth
@pytest.mark.parametrize("path", PATHS)
def test_range_query_dense_hits_regrow(bm, path):
    """Every pair a hit (9M keys): the first hit buffer overflows and the query is redone."""
    X = W.isotropic(3000, 8, 10, seed=21)
    off, ids, st = bm.bm_range_query(torch.from_numpy(X).cuda(), torch.from_numpy(X).cuda(), 1e3, path=path)
    assert ids.numel() == 3000 * 3000
    assert np.array_equal(off.cpu().numpy(), np.arange(3001, dtype=np.int64) * 3000)
    assert np.array_equal(ids.cpu().numpy().reshape(3000, 3000), np.tile(np.arange(3000, dtype=np.int32), (3000, 1)))


@pytest.mark.parametrize("path", PATHS)
def test_build_step_buffer_regrow(bm, path):
    """Large balls: a greedy step produces more hits than the first step buffer holds."""
    X = W.isotropic(20000, 2, 10, seed=22)
    ref = oracle.build(X, 2.0)
    assert_same_graph(run_build(bm, X, 2.0, path), ref)


@pytest.mark.parametrize("path", PATHS)
def test_build_membership_buffer_regrow(bm, path):
    """Cover multiplicity ~6 at n = 200k: the membership keys outgrow their first buffer
    (4n keys) and the greedy grows it and redoes the step, with no restart."""
    X = W.isotropic(200_000, 8, 10, seed=23)
    ref = oracle.build(X, 3.0)
    assert ref["ids"].size > 4 * X.shape[0]
    assert_same_graph(run_build(bm, X, 3.0, path), ref)


# ------------------------------------------------------------------ magnitudes (fp16 scaling)
@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("scale,offset", [(1e4, 3e5), (1e-6, 0.0), (1.0, 1e3), (2.0 ** -30, 2.0 ** -20)])
def test_magnitudes_far_from_one(bm, path, scale, offset):
    """Coordinates far outside [-1, 1] or tiny: the fp16 path scales them by a power
    of two; large offsets make the norms dwarf the distances (wide bands, many
    rechecks); every path must still match the oracle."""
    X = (W.isotropic(3000, 12, 10, seed=31).astype(np.float64) * scale + offset).astype(np.float32)
    D = ((X[:200, None, :].astype(np.float64) - X[None, :, :]) ** 2).sum(-1)
    eps = float(np.sqrt(np.quantile(D[D > 0], 0.002)))
    assert_same_graph(run_build(bm, X, eps, path), oracle.build(X, eps), (scale, offset))
    Q = X[::13]
    off, ids, _ = bm.bm_range_query(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), eps, path=path)
    ro, ri = oracle.range_query(X, Q, eps)
    assert np.array_equal(off.cpu().numpy(), ro) and np.array_equal(ids.cpu().numpy(), ri)


# ------------------------------------------------------------------ automatic path
def test_auto_switches_to_split_on_wide_bands(bm):
    """Swiss roll at d = 128: the fp16 band holds far more pairs than the tiles save,
    so the automatic path moves to the bf16 split during the greedy; same result."""
    X = W.swissroll(30000, 128, 12, seed=3)
    got = run_build(bm, X, 0.6, "auto")
    assert got["stats"]["path"] == bm.BM_PATH_TC_SPLIT3
    assert_same_graph(got, oracle.build(X, 0.6))


def test_auto_stays_fp16_on_separated_data(bm):
    """Well-separated mixture (every ball a singleton): the band stays tiny and the
    automatic path keeps the fp16 tiles for the whole build."""
    X = W.mixture(20000, 64, 8, clusters=32, seed=1)
    got = run_build(bm, X, 4.0, "auto")
    assert got["stats"]["path"] == bm.BM_PATH_TC_FP16
    assert_same_graph(got, oracle.build(X, 4.0))


def test_auto_returns_to_split_when_fp16_band_grows(bm):
    """Norms far larger than eps (offset cloud, tiny eps): the split's band is empty, so
    the automatic path moves to fp16, where every self pair falls into the wider band
    (1/n of the pairs > 2e-4 at n = 3000) and it returns to the split; same result."""
    X = (W.isotropic(3000, 16, 10, seed=8).astype(np.float64) + 50.0).astype(np.float32)
    got = run_build(bm, X, 0.5, "auto")
    assert got["stats"]["path"] == bm.BM_PATH_TC_SPLIT3
    assert_same_graph(got, oracle.build(X, 0.5))
