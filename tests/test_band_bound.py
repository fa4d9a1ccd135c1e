"""The proven error band of the distance tiles (bm_band_halfwidth, Sec. 3.2) against an
emulation of their arithmetic on the CPU.

The tiles compute v = q.x - phi_q - phi_x = (eps^2 - D)/2 from 16-bit operands: the bf16
split (hi = bf16(x), lo = bf16(x - hi), products hi.hi + lo.hi + hi.lo) or fp16 on
coordinates scaled by 2^e, plus an augmentation block carrying three 16-bit pieces of each
side's FP64 phi and the query row's delta'.  Every product is exact in FP32; the
accumulation order and rounding of the tensor cores are not specified, so the emulation
adds the terms in FP32 with rounding toward zero in three orders (K order, reversed, and a
random permutation).  The accumulator must land within the bound of the exact
v + delta', for rows of very different norms, with and without the translation of the
operands by the points' mean, and on inputs built so that the operand roundings all point
the same way (the case the representation terms of the bound are for)."""
import numpy as np
import pytest

from paper_2601_01405_gb300 import _build, binding
from paper_2601_01405_gb300 import workloads as W


@pytest.fixture(scope="module")
def bm():
    _build.build()
    return binding


def round_sig(x, bits):
    """Nearest value with `bits` significant bits (ties to even), in float64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 2.0 ** bits) / 2.0 ** bits, e)


def bf16(x):
    return round_sig(x, 8)


def fp16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def pieces(phi, rnd):
    """Three 16-bit pieces of an FP64 value, each the rounding of what remains."""
    p1 = rnd(phi)
    r1 = phi - p1
    p2 = rnd(r1)
    p3 = rnd(r1 - p2)
    return p1, p2, p3


def f32_toward_zero(s):
    f = np.float32(s)
    if abs(float(f)) > abs(s):
        f = np.nextafter(f, np.float32(0.0))
    return float(f)


def accumulate(terms, order):
    acc = 0.0
    for t in terms[order]:
        acc = f32_toward_zero(acc + float(t))
    return acc


def tile_terms(a, b, phi_a, phi_b, dprime, path, scale_exp):
    """The K terms of one (query, point) accumulator, in K order."""
    if path == "tc":
        ha, hb = bf16(a), bf16(b)
        la, lb = bf16(a - ha), bf16(b - hb)
        prod = np.concatenate([ha * hb, la * hb, ha * lb])
        rnd = bf16
    else:
        sc = 2.0 ** scale_exp
        prod = fp16(a * sc) * fp16(b * sc)
        rnd = fp16
    pa, pb = pieces(phi_a, rnd), pieces(phi_b, rnd)
    aug = np.array([-pa[0], -pa[1], -pa[2], -pb[0], -pb[1], -pb[2], dprime])
    return np.concatenate([prod, aug])


def check_rows(bm, X, Q, eps, path, centre=None, pairs=160, seed=0):
    """Every sampled (q, x) pair: |acc - (v + delta'_q)| <= delta_q for three orders."""
    rng = np.random.default_rng(seed)
    X = np.asarray(X, np.float64)
    Q = np.asarray(Q, np.float64)
    c = np.zeros(X.shape[1]) if centre is None else np.asarray(centre, np.float64)
    Xc = (np.float32(X) - np.float32(c)).astype(np.float64)   # fl(x - c), float32 like the prep kernel
    Qc = (np.float32(Q) - np.float32(c)).astype(np.float64)
    d = X.shape[1]
    d_pad = d
    e2 = eps * eps
    Nb = float(np.sqrt((Xc ** 2).sum(1)).max())
    Na_all = np.sqrt((Qc ** 2).sum(1))
    scale_exp = 0
    if path == "tc16":
        k = int(np.frexp(max(float(max(Nb, Na_all.max())), eps))[1])
        scale_exp = 7 - k
    sc = 2.0 ** scale_exp
    Pb = max(Nb * Nb / 2 - e2 / 4, e2 / 4)
    worst = 0.0
    for _ in range(pairs):
        i = int(rng.integers(Q.shape[0]))
        j = int(rng.integers(X.shape[0]))
        a, b = Qc[i], Xc[j]
        phi_a = (a @ a) / 2 * sc * sc - e2 * sc * sc / 4
        phi_b = (b @ b) / 2 * sc * sc - e2 * sc * sc / 4
        delta = bm.band_halfwidth(path, d, d_pad, Na_all[i] * sc, Nb * sc, abs(phi_a), Pb * sc * sc)
        dprime = (bf16 if path == "tc" else fp16)(delta * (1 + 2 ** -7))   # rounded up is >= delta
        D = float(((Q[i] - X[j]) ** 2).sum())                              # the untranslated exact distance
        v = (e2 - D) / 2 * sc * sc
        terms = tile_terms(a, b, phi_a, phi_b, dprime, path, scale_exp)
        T = v + dprime
        K = len(terms)
        for order in (np.arange(K), np.arange(K)[::-1], rng.permutation(K)):
            err = abs(accumulate(terms, order) - T)
            assert err <= delta, (path, i, j, err, delta)
            worst = max(worst, err / delta)
    return worst


@pytest.mark.parametrize("path", ["tc", "tc16"])
def test_band_holds_on_varied_norms(bm, path):
    """Queries from near the origin to far out against a cloud: each row's own bound."""
    X = W.isotropic(3000, 64, 10, seed=61) * np.float32(3.0)
    Q = np.concatenate([X[:40] * np.float32(0.01), X[40:80], X[80:120] * np.float32(4.0)])
    check_rows(bm, X, Q, 6.0, path)


@pytest.mark.parametrize("path", ["tc", "tc16"])
def test_band_holds_on_translated_operands(bm, path):
    """A cloud far from the origin, its operands translated by the mean; the distances the
    accumulator approximates are those of the untranslated rows."""
    X = (W.isotropic(2000, 32, 10, seed=62).astype(np.float64) + 25.0).astype(np.float32)
    check_rows(bm, X, X[::13], 3.0, path, centre=X.mean(0))
    check_rows(bm, X, X[::13], 3.0, path)   # and untranslated


def test_band_holds_on_the_roll(bm):
    X = W.swissroll(4000, 128, 12, seed=63)
    check_rows(bm, X, X[::17], 0.5, "tc", centre=X.astype(np.float64).mean(0))


@pytest.mark.parametrize("path", ["tc", "tc16"])
def test_band_holds_when_every_rounding_points_the_same_way(bm, path):
    """Coordinates just below a rounding boundary of the 16-bit type, all positive: every
    operand rounds up by almost half a unit, so the representation error of q.x is as large
    as it gets and of one sign; the bound must still hold (a bound without its
    representation term would not)."""
    bits = 8 if path == "tc" else 11
    rng = np.random.default_rng(64)
    k = rng.integers(0, 6, size=(64, 48))
    x = (1.0 + (2.0 * rng.integers(0, 2 ** (bits - 2), size=(64, 48)) + 1.0 - 2.0 ** -6) * 2.0 ** (-bits)) * 2.0 ** k
    X = x.astype(np.float32)
    worst = check_rows(bm, X, X, 4.0, path, pairs=120, seed=3)
    if path == "tc16":
        # about a third of the bound is reached: the fp16 bound is almost all representation
        # term (2^-10 N_a N_b), so a bound without it (some 30 times smaller) fails here
        assert worst > 0.1
    else:
        assert worst > 0.0


@pytest.mark.parametrize("path", ["tc", "tc16", "fp32"])
def test_band_grows_with_the_norms_and_the_row_bound_is_below_the_maximum(bm, path):
    """Monotone in every magnitude, so a row's own bound never exceeds the bound of the
    largest norm and |phi| (what lets the tiles use one offset per row)."""
    base = bm.band_halfwidth(path, 64, 64, 10.0, 20.0, 50.0, 200.0)
    assert base > 0.0
    for args in ((11.0, 20.0, 50.0, 200.0), (10.0, 21.0, 50.0, 200.0), (10.0, 20.0, 60.0, 200.0),
                 (10.0, 20.0, 50.0, 210.0)):
        assert bm.band_halfwidth(path, 64, 64, *args) > base
    assert bm.band_halfwidth(path, 64, 128, 10.0, 20.0, 50.0, 200.0) >= base   # more K terms
