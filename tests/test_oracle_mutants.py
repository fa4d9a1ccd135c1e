"""Plant plausible mistakes in a copy of the oracle's C source and check that every
one of them trips at least one pin (a dropped term, a wrong sign, a wrong index,
a transposed operand, a non-strict comparison, a broken greedy).  Runs on the
CPU only; the real oracle is never modified."""
import os
import tempfile

import pytest

import oracle
import pins
from paper_2601_01405_gb300 import workloads as W

SRC = os.path.join(os.path.dirname(oracle.__file__), "bm_oracle.c")

# (name, original text, replacement, count of replacements expected or None for all)
MUTANTS = [
    ("closed-ball", "< eps2", "<= eps2", None),
    ("dropped-last-term", "for (int i = 0; i < d; ++i) {\n        double t = a[i] - b[i];",
     "for (int i = 0; i + 1 < d; ++i) {\n        double t = a[i] - b[i];", 1),
    ("wrong-sign", "double t = a[i] - b[i];", "double t = a[i] + b[i];", 1),
    ("greedy-ignores-cover", "if (covered[x]) continue;", "if (0) continue;", 1),
    ("greedy-covers-self-only", "< eps2) covered[y] = 1;", "< eps2) covered[y] = (y == x);", 1),
    ("edge-always", "if (a[p] == b[q]) return 1;", "if (a[p] != b[q]) return 1;", 1),
    ("edge-self-loop", "for (int64_t j = i + 1; j < L; ++j) {", "for (int64_t j = i; j < L; ++j) {", 1),
    ("transposed-range-id", "ids[o++] = (int32_t)i;", "ids[o++] = (int32_t)j;", 2),
    ("over-pruned-edges", "4.0 * eps2", "1.0 * eps2", 1),
    ("kth-off-by-one", "kth_smallest(row, n, k - 1)", "kth_smallest(row, n, k)", 1),
    ("balltree-prune-sign", "if (dc - nd->radius > r", "if (dc + nd->radius > r", 1),
    ("balltree-radius-min", "if (s > r2) { r2 = s; pa = p; }", "if (s < r2) { r2 = s; pa = p; }", 1),
    ("balltree-leaf-closed", "t->d) < r2) {", "t->d) <= r2) {", 1),
    ("pair-roles-swapped", "sqdist(Q + (size_t)qrow[k] * d, X + (size_t)xcol[k] * d, d)",
     "sqdist(X + (size_t)qrow[k] * d, Q + (size_t)xcol[k] * d, d)", 1),
    ("fps-ties-to-largest", "if (m[x] > m[best]) best = x;", "if (m[x] >= m[best]) best = x;", 1),
    ("fps-strict-eps", "if (!(m[best] >= eps2)) break;", "if (!(m[best] > eps2)) break;", 1),
    ("fps-no-update", "if (D < m[x]) m[x] = D;", "if (D < m[x] && cur == first) m[x] = D;", 1),
    ("color-mean-divisor", "out[r] = sum / (double)cnt;", "out[r] = sum / (double)(cnt + 1);", 1),
    ("color-median-index", "(v[cnt / 2 - 1] + v[cnt / 2]) / 2.0", "(v[cnt / 2] + v[cnt / 2]) / 2.0", 1),
    ("color-min-max-swapped", "if (stat == 2 ? x < best : x > best)", "if (stat == 2 ? x > best : x < best)", 1),
    ("graph-ties-to-larger-id", "return a.D < b.D || (a.D == b.D && a.id < b.id);",
     "return a.D < b.D || (a.D == b.D && a.id > b.id);", 1),
    ("knn-graph-keeps-self", "if (j == i) continue;", "if (0) continue;", 1),
    ("graph-no-range-expansion", "if (!(w->vd[h] < eps2) || w->expd[h]) continue;", "if (1) continue;", 1),
    ("graph-beam-never-evicts", "if (nR < ef || dkey_less(k, w->R[nR - 1])) {", "if (nR < ef) {", 1),
    ("graph-entry-ignores-distance", "if (D < bd || (D == bd && e < start)) { bd = D; start = e; }",
     "if (t == 0) { bd = D; start = e; }", 1),
    ("masked-ignores-cells", "if (flag[cell_of[i]] && sqdist", "if ((flag[cell_of[i]] || 1) && sqdist", 2),
]
# A wrong node centre is not listed: any centre paired with the radius measured
# from it still bounds the node, so the range sets stay exact.


def _all_pins():
    pins.pin_line()
    pins.pin_grid()
    pins.pin_degenerate()
    pins.pin_brute(seeds=range(25))
    X = W.isotropic(600, 8, 10, seed=1)
    pins.pin_fixpoint(X, 2.5)
    pins.pin_invariants(X, 2.5)
    pins.pin_witness(W.isotropic(300, 8, 10, seed=4), 3.0)
    pins.pin_prune(W.isotropic(800, 16, 10, seed=5), 3.0)
    pins.pin_balltree(W.isotropic(3000, 4, 10, seed=6), 0.5)
    G = W.tiny_grid_cloud(3000, 3, 2, span=8, seed=11)
    pins.pin_balltree(G, 1.0, Q=G[:300])
    pins.pin_knn_scipy(W.paper_gaussian_fp64(500, 6, seed=7), 20)
    pins.pin_range_scipy(W.paper_gaussian_fp64(800, 5, seed=8), W.paper_gaussian_fp64(800, 5, seed=8)[:50], 1.3)
    pins.pin_pair_sqdist(W.isotropic(300, 16, 10, seed=9), W.isotropic(77, 16, 10, seed=10) * 3, 10)
    pins.pin_masked()
    pins.pin_fps_golden()
    pins.pin_fps_invariants(W.isotropic(600, 5, 10, seed=61), 1.7)
    pins.pin_fps_brute(seeds=range(6))
    pins.pin_color_golden()
    pins.pin_color_lipschitz(W.isotropic(800, 5, 10, seed=63), 1.2)
    pins.pin_color_values(W.isotropic(600, 4, 10, seed=64), 0.9)
    pins.pin_graph_golden()
    pins.pin_knn_graph_scipy(W.paper_gaussian_fp64(500, 5, seed=81), 7)
    Xg = W.isotropic(1200, 6, 10, seed=82)
    pins.pin_graph_exhaustive_and_conservative(Xg, Xg[::29], 1.6)


def test_unmutated_oracle_passes_all_pins():
    _all_pins()


@pytest.mark.parametrize("name,old,new,count", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, count, monkeypatch):
    src = open(SRC).read()
    occurrences = src.count(old)
    assert occurrences >= 1, "mutation site vanished: %s" % name
    if count is not None:
        assert occurrences == count, (name, occurrences)
    mutated = src.replace(old, new)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "mutant.c")
        with open(path, "w") as f:
            f.write(mutated)
        lib = oracle.load_library(oracle.compile_library(force=True, src=path,
                                                         out=os.path.join(tmp, "libmutant.so")))
        monkeypatch.setattr(oracle, "_lib", lib)
        caught = False
        try:
            _all_pins()
        except (AssertionError, ValueError, RuntimeError):
            caught = True
        assert caught, "planted mistake '%s' passed every pin" % name
