"""Farthest-point landmarks (Sec. 2.2) and coloring (Sec. 2.3) on the GPU, through the
C-ABI, against the CPU oracle.

FPS landmarks, their order, memberships and edges are index results: bit-identical
to the oracle.  Median, minimum and maximum colorings select existing values: exact.
The mean is an FP64 sum whose order is unspecified: within (m - 1) 2^-53 sum |f| of
the oracle's sequential sum on each side, plus the division's rounding."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2601_01405_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def bm():
    from paper_2601_01405_gb300 import _build, binding
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def host(out):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


def same_graph(got, ref, tag=""):
    assert np.array_equal(got["landmarks"], ref["landmarks"]), ("landmarks", tag)
    assert np.array_equal(got["offsets"], ref["offsets"]), ("offsets", tag)
    assert np.array_equal(got["ids"], ref["ids"]), ("ids", tag)
    assert np.array_equal(got["edges"].reshape(-1, 2), ref["edges"].reshape(-1, 2)), ("edges", tag)


def fps(bm, X, eps, first=0, path="auto"):
    out = bm.bm_build_fps(torch.from_numpy(np.ascontiguousarray(X)).cuda(), eps, first, path=path)
    torch.cuda.synchronize()
    return host(out)


def test_fps_golden_cases(bm):
    with open(os.path.join(GOLDEN, "fps_line.json")) as fh:
        g = json.load(fh)
    for case in g["cases"]:
        X = W.line_points(10) if case["points"] == "line" else W.grid_points(3)
        out = fps(bm, X, case["eps"], case["first"])
        assert out["landmarks"].tolist() == case["landmarks"], case
        rows = [out["ids"][out["offsets"][i]:out["offsets"][i + 1]].tolist() for i in range(len(case["landmarks"]))]
        assert rows == case["members"], case
        assert out["edges"].tolist() == case["edges"], case


@pytest.mark.parametrize("path", ["auto", "tc", "fp32"])
def test_fps_iso_n10k_d16(bm, path):
    X = W.make("iso-n10k-d16")
    out = fps(bm, X, 3.0, 0, path)
    same_graph(out, oracle.fps_build(X, 3.0, 0))
    assert out["stats"]["greedy_steps"] == out["landmarks"].size


@pytest.mark.parametrize("name,eps,first", [("mix32-n32k-d64", 11.0, 5), ("roll-n50k-d128", 2.0, 49_999),
                                            ("iso-n20k-d128", 14.0, 123)])
def test_fps_reduced_workloads(bm, name, eps, first):
    X = W.make(name)
    same_graph(fps(bm, X, eps, first), oracle.fps_build(X, eps, first), name)


def test_fps_ties_and_degenerate(bm):
    G = W.tiny_grid_cloud(3000, 3, 1, span=5, seed=71)      # many exact ties at eps
    for eps in (1.0, 1.5, 2.0):
        same_graph(fps(bm, G, eps, 7), oracle.fps_build(G, eps, 7), eps)
    same_graph(fps(bm, np.full((50, 4), 1.5, dtype=np.float32), 0.1), oracle.fps_build(
        np.full((50, 4), 1.5, dtype=np.float32), 0.1))      # all identical: one landmark
    same_graph(fps(bm, W.isotropic(1, 3, 10, seed=72), 1.0), oracle.fps_build(W.isotropic(1, 3, 10, seed=72), 1.0))
    X = W.isotropic(400, 5, 10, seed=73)                    # eps below every gap: all points
    out = fps(bm, X, 1e-4, 3)
    assert out["landmarks"].size == 400
    same_graph(out, oracle.fps_build(X, 1e-4, 3))


def test_fps_host_io_and_errors(bm):
    X = W.isotropic(2000, 7, 10, seed=74)
    out = bm.bm_build_fps(X, 2.0, 11)
    same_graph(out, oracle.fps_build(X, 2.0, 11))
    Xd = torch.from_numpy(X).cuda()
    for bad in (-1, 2000):
        with pytest.raises(bm.BallMapperError) as ei:
            bm.bm_build_fps(Xd, 2.0, bad)
        assert ei.value.status == bm.BM_ERR_ARG
    Xn = Xd.clone()
    Xn[5, 5] = float("inf")
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_build_fps(Xn, 2.0, 0)
    assert ei.value.status == bm.BM_ERR_ARG


# ---------------------------------------------------------------- coloring
def mean_tolerance(off, ids, f):
    absf = np.abs(f.astype(np.float64))
    out = np.empty(off.size - 1)
    for i in range(off.size - 1):
        m = off[i + 1] - off[i]
        s = absf[ids[off[i]:off[i + 1]]].sum()
        out[i] = 2.0 * max(m - 1, 0) * 2.0 ** -53 * s / max(m, 1) + 4.0 * 2.0 ** -53 * s / max(m, 1)
    return out


@pytest.mark.parametrize("name,eps", [("iso-n10k-d16", 3.0), ("mix32-n32k-d64", 11.0), ("iso-n20k-d128", 14.0)])
@pytest.mark.parametrize("stat", ["mean", "median", "min", "max"])
def test_color_matches_oracle(bm, name, eps, stat):
    X = W.make(name)
    Xd = torch.from_numpy(X).cuda()
    g = bm.bm_build(Xd, eps)
    rng = np.random.default_rng(75)
    f = (rng.standard_normal(X.shape[0]) * 3.0).astype(np.float32)
    got = bm.bm_color(g["offsets"], g["ids"], torch.from_numpy(f).cuda(), stat)
    torch.cuda.synchronize()
    off, ids = g["offsets"].cpu().numpy(), g["ids"].cpu().numpy()
    ref = oracle.color(off, ids, f, stat)
    got = got.cpu().numpy()
    if stat == "mean":
        assert np.all(np.abs(got - ref) <= mean_tolerance(off, ids, f))
    else:
        assert np.array_equal(got, ref)


def test_color_golden_and_host_io(bm):
    with open(os.path.join(GOLDEN, "color_line.json")) as fh:
        g = json.load(fh)
    X = W.line_points(10)
    b = bm.bm_build(X, g["eps"])
    f = (X[:, 0].astype(np.float64) ** 2).astype(np.float32)
    for stat in ("mean", "median", "min", "max"):
        got = bm.bm_color(b["offsets"], b["ids"], f, stat)
        assert np.abs(got - np.array(g[stat])).max() <= 1e-14 * 81, stat


def test_color_lipschitz_on_gpu_colorings(bm):
    """Sec. 2.3 bounds that hold for colorings between a ball's min and max, f = k <w, x>:
    |c_i - f(l_i)| < k eps, within a ball < 2 k eps, across an edge < 4 k eps."""
    X = W.make("iso-n10k-d16")
    k, eps = 2.0, 3.0
    w = np.random.default_rng(76).standard_normal(16)
    w /= np.linalg.norm(w)
    f64 = k * (X.astype(np.float64) @ w)
    f = f64.astype(np.float32)                       # the float the GPU colors; Lipschitz up to rounding
    out = host(bm.bm_build(torch.from_numpy(X).cuda(), eps))
    lm, off, ids, E = out["landmarks"], out["offsets"], out["ids"], out["edges"]
    slack = 1e-5 * k * eps
    for stat in ("mean", "median", "min", "max"):
        c = bm.bm_color(torch.from_numpy(off).cuda(), torch.from_numpy(ids).cuda(), torch.from_numpy(f).cuda(),
                        stat).cpu().numpy()
        assert np.all(np.abs(c - f[lm]) < k * eps + slack)
        for i in range(lm.size):
            row = f[ids[off[i]:off[i + 1]]].astype(np.float64)
            assert row.min() <= c[i] <= row.max()
            assert np.abs(row - c[i]).max() < 2 * k * eps + slack
        if E.size:
            assert np.abs(c[E[:, 0]] - c[E[:, 1]]).max() < 4 * k * eps + slack


def test_color_errors_and_empty_rows(bm):
    off = torch.tensor([0, 2, 2, 3], dtype=torch.int64, device="cuda")
    ids = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda")
    f = torch.tensor([1.0, 2.0, 4.0], dtype=torch.float32, device="cuda")
    c = bm.bm_color(off, ids, f, "mean").cpu().numpy()
    assert c[0] == 1.5 and np.isnan(c[1]) and c[2] == 4.0
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_color(off, torch.tensor([0, 1, 3], dtype=torch.int32, device="cuda"), f, "max")
    assert ei.value.status == bm.BM_ERR_ARG
    with pytest.raises(bm.BallMapperError) as ei:
        bm.bm_color(off, ids, torch.tensor([1.0, float("nan"), 4.0], device="cuda"), "median")
    assert ei.value.status == bm.BM_ERR_ARG
