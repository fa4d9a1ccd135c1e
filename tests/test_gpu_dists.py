"""Reported distances (bm_csr.dists, opt.want_dists) against the CPU oracle, element by
element.

Every stored pair (row, point) of a membership or range-query CSR carries d(q_row, x)
as a float.  The bar is a relative error of at most 1e-6 against the oracle's FP64
distance sqrt(D), D the FP64 squared distance summed in coordinate order
(oracle.pair_sqdist).  The library computes D with that same arithmetic and rounds
sqrt(D) once to float, so its error is at most 2^-24 and the per-run figure it reports
(stats.dist_max_rel_err) must agree with the one measured here."""
import numpy as np
import pytest

import oracle
from paper_2601_01405_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-6
PATHS = ["auto", "tc", "tc16", "fp32"]


@pytest.fixture(scope="module")
def bm():
    from paper_2601_01405_gb300 import _build, binding
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def rel_err(got, X, Q, rows_q, ids):
    """Relative error of got against the oracle's FP64 sqrt(D(Q[rows_q], X[ids]))."""
    ref = np.sqrt(oracle.pair_sqdist(X, Q, rows_q.astype(np.int32), ids.astype(np.int32)))
    g = got.astype(np.float64)
    err = np.where(ref > 0, np.abs(g - ref) / np.where(ref > 0, ref, 1.0), np.abs(g))
    return err, ref


def check_csr(off, ids, dists, stats, X, Q):
    off, ids, dists = (np.asarray(a) for a in (off, ids, dists))
    assert dists.dtype == np.float32 and dists.size == ids.size
    rows = np.repeat(np.arange(off.size - 1), np.diff(off))
    err, ref = rel_err(dists, X, Q, rows, ids)
    assert err.max(initial=0.0) <= REL_TOL, err.max()
    # the reported figure is the error actually made (same FP64 value on both sides)
    assert abs(stats["dist_max_rel_err"] - err.max(initial=0.0)) <= 1e-12
    assert stats["dist_max_rel_err"] <= 2.0 ** -24
    # the float nearest to the FP64 distance, entry by entry
    assert np.array_equal(dists, ref.astype(np.float32))


@pytest.mark.parametrize("path", PATHS)
def test_build_dists_iso_n10k_d16(bm, path):
    X = W.make("iso-n10k-d16")
    out = bm.bm_build(torch.from_numpy(X).cuda(), 3.0, path=path, want_dists=True)
    torch.cuda.synchronize()
    ref = oracle.build(X, 3.0)
    lm = out["landmarks"].cpu().numpy()
    assert np.array_equal(lm, ref["landmarks"])
    off, ids = out["offsets"].cpu().numpy(), out["ids"].cpu().numpy()
    assert np.array_equal(ids, ref["ids"])
    # rows are balls around landmarks: the query of row r is X[lm[r]]
    check_csr(off, ids, out["dists"].cpu().numpy(), out["stats"], X, X[lm])
    st = out["stats"]
    assert st["recheck_rate"] == pytest.approx(st["band_pairs"] / st["tile_pairs"])


@pytest.mark.parametrize("path", PATHS)
def test_range_dists_on_tie_heavy_grid(bm, path):
    """Integer-grid cloud: many pairs at exactly eps (excluded) and at distance 0."""
    X = W.tiny_grid_cloud(6000, 3, 2, span=8, seed=41)
    Q = X[:700]
    off, ids, st, dists = bm.bm_range_query(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), 1.0,
                                            path=path, want_dists=True)
    torch.cuda.synchronize()
    ro, ri = oracle.range_query(X, Q, 1.0)
    assert np.array_equal(off.cpu().numpy(), ro) and np.array_equal(ids.cpu().numpy(), ri)
    d = dists.cpu().numpy()
    assert np.all(d < 1.0) and np.any(d == 0.0)
    check_csr(ro, ri, d, st, X, Q)


@pytest.mark.parametrize("scale,offset", [(1e4, 3e5), (1e-6, 0.0), (2.0 ** -30, 2.0 ** -20), (1e15, 0.0)])
def test_dists_extreme_magnitudes(bm, scale, offset):
    X = (W.isotropic(2500, 12, 10, seed=43).astype(np.float64) * scale + offset).astype(np.float32)
    D = ((X[:200, None, :].astype(np.float64) - X[None, :, :]) ** 2).sum(-1)
    eps = float(np.sqrt(np.quantile(D[D > 0], 0.004)))
    Q = X[::7]
    off, ids, st, dists = bm.bm_range_query(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), eps,
                                            want_dists=True)
    torch.cuda.synchronize()
    ro, ri = oracle.range_query(X, Q, eps)
    assert np.array_equal(ids.cpu().numpy(), ri)
    check_csr(ro, ri, dists.cpu().numpy(), st, X, Q)


def test_dists_host_io_and_queries_off_the_points(bm):
    X = W.mixture(9000, 40, 8, clusters=9, seed=44)
    # queries near the points but not on them
    Q = (X[::27][:333] + W.isotropic(333, 40, 8, seed=45) * np.float32(0.5)).astype(np.float32)
    off, ids, st, dists = bm.bm_range_query(X, Q, 9.0, want_dists=True)
    assert isinstance(dists, np.ndarray)
    ro, ri = oracle.range_query(X, Q, 9.0)
    assert np.array_equal(off, ro) and np.array_equal(ids, ri) and ri.size > 0
    check_csr(ro, ri, dists, st, X, Q)
    g = bm.bm_build(X, 9.0, want_dists=True)
    check_csr(g["offsets"], g["ids"], g["dists"], g["stats"], X, X[g["landmarks"]])


def test_dists_through_the_inverted_file(bm):
    X = W.make("iso-n20k-d128")
    Xd = torch.from_numpy(X).cuda()
    idx = bm.IvfIndex(Xd, nlist=64, iters=8, seed=3)
    Q = Xd[:500].contiguous()
    off, ids, probes, st, dists = idx.range_query(Q, 14.0, 8, want_dists=True)
    torch.cuda.synchronize()
    check_csr(off.cpu().numpy(), ids.cpu().numpy(), dists.cpu().numpy(), st, X, X[:500])
    g = idx.build(14.0, 8, want_dists=True)
    torch.cuda.synchronize()
    lm = g["landmarks"].cpu().numpy()
    check_csr(g["offsets"].cpu().numpy(), g["ids"].cpu().numpy(), g["dists"].cpu().numpy(), g["stats"], X, X[lm])


def test_batched_rejects_want_dists(bm):
    from paper_2601_01405_gb300 import binding
    lib = binding.load()
    X = torch.zeros((10, 2), dtype=torch.float32, device="cuda")
    inst = (binding.bm_instance * 1)()
    inst[0].X, inst[0].n, inst[0].d, inst[0].eps = X.data_ptr(), 10, 2, 1.0
    opt = binding.bm_options()
    lib.bm_options_init(opt)
    opt.want_dists = 1
    outs = (binding.bm_graph * 1)()
    assert lib.bm_build_batched(inst, 1, opt, outs, None) == binding.BM_ERR_ARG
