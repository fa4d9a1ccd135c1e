"""The CPU oracle against facts fixed by the paper and by mathematics (no GPU)."""
import numpy as np
import pytest

import oracle
import pins
from paper_2601_01405_gb300 import workloads as W


def test_line_golden():
    pins.pin_line()


def test_grid_golden():
    pins.pin_grid()


def test_degenerate_cases():
    pins.pin_degenerate()


def test_tiny_brute_force_rational():
    pins.pin_brute()


@pytest.mark.parametrize("name,eps", [("iso", 3.0), ("mix", 11.0), ("roll", 1.0)])
def test_fixpoint_and_invariants(name, eps):
    if name == "iso":
        X = W.isotropic(1500, 16, 10, seed=1)
    elif name == "mix":
        X = W.mixture(1024, 64, 8, clusters=32, seed=2)
    else:
        X = W.swissroll(1500, 128, 12, seed=3)
    pins.pin_fixpoint(X, eps)
    pins.pin_invariants(X, eps)


@pytest.mark.parametrize("eps", [2.0, 3.0, 4.5])
def test_witness_radius(eps):
    X = W.isotropic(400, 8, 10, seed=4)
    pins.pin_witness(X, eps)


def test_edge_pruning_is_exact():
    pins.pin_prune(W.isotropic(2000, 16, 10, seed=5), 3.0)
    pins.pin_prune(W.swissroll(2000, 128, 12, seed=6), 1.0)


def test_balltree_iso_n10k_d16():
    X = W.make("iso-n10k-d16")
    pins.pin_balltree(X, 3.0)


def test_balltree_roll_subsample():
    X = W.swissroll(20000, 128, 12, seed=0)
    pins.pin_balltree(X, 1.0)


def test_balltree_ties_on_grid():
    X = W.tiny_grid_cloud(3000, 3, 2, span=8, seed=11)
    pins.pin_balltree(X, 1.0, Q=X[:500])


def test_knn_against_scipy():
    pins.pin_knn_scipy(W.paper_gaussian_fp64(2000, 10, seed=7), 50)


def test_range_against_scipy():
    X = W.paper_gaussian_fp64(3000, 5, seed=8)
    pins.pin_range_scipy(X, X[:200], 1.3)


def test_masked_range_query():
    pins.pin_masked()


def test_pair_sqdist():
    pins.pin_pair_sqdist(W.isotropic(300, 16, 10, seed=9), W.isotropic(77, 16, 10, seed=10) * 3, 10)


def test_iso_n10k_d16_counts():
    """The 10k x 16 isotropic workload at eps = 3: landmark count, membership count
    and edge count of the exact Ball Mapper, cross-checked by the invariants."""
    X = W.make("iso-n10k-d16")
    out = oracle.build(X, 3.0)
    assert np.all(np.diff(out["landmarks"]) > 0)
    assert out["offsets"][-1] == out["ids"].size
    pins.pin_fixpoint(X[:3000], 3.0)


@pytest.mark.slow
def test_paper_worked_example():
    """Sec. 6.3: Gaussian n=20000, d=50, k=50 -> eps ~ 7.5536, 6361 landmarks, 936690 edges."""
    pins.pin_paper()


def test_fps_golden_line_and_grid():
    pins.pin_fps_golden()


def test_fps_invariants_and_brute_force():
    pins.pin_fps_invariants(W.isotropic(1500, 6, 10, seed=61), 1.7)
    pins.pin_fps_invariants(W.tiny_grid_cloud(800, 2, 1, span=6, seed=62), 1.0, first=17)
    pins.pin_fps_brute()


def test_color_golden_line():
    pins.pin_color_golden()


def test_color_lipschitz_bounds_and_values():
    pins.pin_color_lipschitz(W.isotropic(2000, 5, 10, seed=63), 1.2)
    pins.pin_color_values(W.isotropic(1500, 4, 10, seed=64), 0.9)


def test_paper_coloring_bound_needs_the_diameter():
    """Sec. 2.3, Prop. 2.4 as printed (max |f(x) - c(l_i)| <= k eps) fails for the mean on a
    lopsided ball: f(x) = x (k = 1), landmark 0, eps = 1, members {-0.9, 0, 0.9, 0.9, 0.9}
    give c = 0.36 and |f(-0.9) - c| = 1.26 > 1.  The bound that holds is 2 k eps."""
    X = np.array([[0.0], [-0.875], [0.875], [0.875], [0.875]], dtype=np.float32)
    out = oracle.build(X, 1.0)
    assert out["landmarks"].tolist() == [0]
    c = oracle.color(out["offsets"], out["ids"], X[:, 0], "mean")[0]
    assert abs(-0.875 - c) > 1.0 and abs(-0.875 - c) < 2.0


def test_graph_oracle_golden():
    pins.pin_graph_golden()


def test_knn_graph_against_scipy():
    pins.pin_knn_graph_scipy(W.paper_gaussian_fp64(1500, 7, seed=81), 9)


def test_graph_oracle_exhaustive_and_conservative():
    X = W.isotropic(2400, 6, 10, seed=82)
    pins.pin_graph_exhaustive_and_conservative(X, X[::37], 1.6)
