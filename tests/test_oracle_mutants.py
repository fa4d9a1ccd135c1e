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
