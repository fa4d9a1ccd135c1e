"""Full-size workloads in the configuration bench.py times, checked against the CPU
oracle on sampled outputs (each sampled value computed by the oracle one by one) and
through properties that hold at any size."""
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


def sampled_checks(X, out, eps, rng, n_points=400, n_rows=120, n_edges=200):
    """X: host float32 points; out: bm_build result as device tensors (large arrays stay
    on the device; only sampled rows come to the host)."""
    n = X.shape[0]
    lm = out["landmarks"].cpu().numpy()
    off = out["offsets"].cpu().numpy()
    ids_d, edges_d = out["ids"], out["edges"]
    L = lm.size
    # landmarks strictly increasing; every point covered; each row non-empty, ascending, unique
    assert L >= 1 and np.all(np.diff(lm) > 0)
    assert int(torch.bincount(ids_d.long(), minlength=n).min()) >= 1
    assert off[0] == 0 and off[-1] == ids_d.numel() and np.all(np.diff(off) >= 1)
    row_of = torch.repeat_interleave(torch.arange(L, device=ids_d.device),
                                     torch.from_numpy(np.diff(off)).to(ids_d.device))
    asc = (ids_d[1:] > ids_d[:-1]) | (row_of[1:] != row_of[:-1])
    assert bool(asc.all())
    # index-order greedy characterisation on sampled points:
    # x is a landmark  <=>  no landmark l < x has d(l, x) < eps
    xs = np.unique(np.concatenate([rng.integers(0, n, n_points), lm[rng.integers(0, L, 50)]]))
    lo, li = oracle.range_query(X[lm], X[xs], eps)
    is_lm = np.isin(xs, lm)
    for k, x in enumerate(xs):
        covered_earlier = np.any(lm[li[lo[k]:lo[k + 1]]] < x)
        assert is_lm[k] == (not covered_earlier), x
    # membership rows of sampled landmarks: full-scan oracle rows
    rows = np.unique(rng.integers(0, L, n_rows))
    ro, ri = oracle.range_query(X, X[lm[rows]], eps)
    for k, r in enumerate(rows):
        assert np.array_equal(ids_d[off[r]:off[r + 1]].cpu().numpy(), ri[ro[k]:ro[k + 1]]), r
    E = edges_d.shape[0]
    ekeys = edges_d[:, 0].long() * L + edges_d[:, 1].long() if E else None
    if E:
        assert bool((edges_d[:, 0] < edges_d[:, 1]).all())
        assert bool((ekeys[1:] > ekeys[:-1]).all())            # lexicographic, unique
        # sampled edges: both balls (oracle rows) share a point
        es = edges_d[torch.from_numpy(rng.integers(0, E, min(n_edges, E))).to(edges_d.device)].cpu().numpy()
        eo, ei = oracle.range_query(X, X[lm[es.ravel()]], eps)
        for k in range(es.shape[0]):
            a = ei[eo[2 * k]:eo[2 * k + 1]]
            b = ei[eo[2 * k + 1]:eo[2 * k + 2]]
            assert np.intersect1d(a, b).size > 0, es[k]
    # sampled landmark pairs closer than 2 eps: an edge exactly when the balls share a point
    cand = rng.integers(0, L, (600, 2))
    cand = cand[cand[:, 0] < cand[:, 1]]
    d2 = ((X[lm[cand[:, 0]]].astype(np.float64) - X[lm[cand[:, 1]]]) ** 2).sum(1)
    close = cand[d2 < 4.0 * float(eps) ** 2][:60]
    if close.shape[0]:
        co, ci = oracle.range_query(X, X[lm[close.ravel()]], eps)
        q = torch.from_numpy(close[:, 0].astype(np.int64) * L + close[:, 1]).to(ids_d.device)
        if E:
            pos = torch.searchsorted(ekeys, q).clamp(max=E - 1)
            present = (ekeys[pos] == q).cpu().numpy()
        else:
            present = np.zeros(close.shape[0], dtype=bool)
        for k in range(close.shape[0]):
            shared = np.intersect1d(ci[co[2 * k]:co[2 * k + 1]], ci[co[2 * k + 1]:co[2 * k + 2]]).size > 0
            assert shared == bool(present[k]), close[k]


def run(bm, Xd, eps, path="tc"):
    out = bm.bm_build(Xd, eps, path=path)
    torch.cuda.synchronize()
    return out


@pytest.fixture(scope="module")
def mix():
    return W.make("mix32-n1M-d64")


# the automatic path (the one bench.py times) at every eps of the workload, and the two
# fixed tensor-core representations at one eps each
@pytest.mark.parametrize("eps,path", [(2.0, "auto"), (4.0, "auto"), (6.0, "auto"), (2.0, "tc16"), (4.0, "tc")])
def test_mix32_n1M_d64_sampled(bm, mix, eps, path):
    Xd = torch.from_numpy(mix).cuda()
    out = run(bm, Xd, eps, path)
    sampled_checks(mix, out, eps, np.random.default_rng(int(eps)))


def test_mix32_n1M_d64_paths_identical(bm, mix):
    """All distance-tile paths give the same bytes at full size (eps = 6)."""
    Xd = torch.from_numpy(mix).cuda()
    a = run(bm, Xd, 6.0, "tc")
    for other in ("fp32", "tc16", "auto"):
        b = run(bm, Xd, 6.0, other)
        for k in ("landmarks", "offsets", "ids", "edges"):
            assert torch.equal(a[k], b[k]), (other, k)


@pytest.mark.parametrize("eps", [0.5, 1.0])
def test_roll_n2M_d128_sampled(bm, eps):
    X = W.make("roll-n2M-d128")
    out = run(bm, torch.from_numpy(X).cuda(), eps)
    sampled_checks(X, out, eps, np.random.default_rng(7 + int(10 * eps)), n_points=200, n_rows=60)


def test_iso_n1M_d128_sampled(bm):
    """The dense-ball workload at eps = 14: 70,430 landmarks, 67.5M memberships, about
    1.2e10 witnessed landmark pairs reduced to the nerve edges in landmark-range chunks."""
    X = W.make("iso-n1M-d128")
    out = run(bm, torch.from_numpy(X).cuda(), 14.0)
    assert out["stats"]["edge_pairs"] > (1 << 32)      # more than one sort's worth: chunked
    sampled_checks(X, out, 14.0, np.random.default_rng(14), n_points=300, n_rows=60, n_edges=100)
