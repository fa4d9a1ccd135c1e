"""Seeded synthetic point clouds shaped like the paper's workloads.

This module only draws and quantises coordinates; it holds none of the Ball
Mapper arithmetic, so both the CPU oracle (tests) and the CUDA path consume
the very same bytes from it.

The paper evaluates on synthetic isotropic, clustered and low-dimensional
structured point clouds in R^d with the Euclidean distance (Sec. 6.1).  Its
generator parameters are not printed, so the recipes below fix them:

* ``isotropic``  X ~ N(0, I_d)
* ``mixture``    equal-weight clusters, centres uniform in [-10, 10]^d,
                 isotropic sigma = 1, labels shuffled so index order is random
* ``swissroll``  t ~ U[1.5 pi, 4.5 pi], h ~ U[0, 20], P = (t cos t, h, t sin t)
                 mapped into R^d by a seeded orthonormal 3-frame, plus
                 N(0, 0.01^2) noise in every coordinate
* ``batched``    many independent isotropic / 8-cluster instances of uneven n

Coordinates are quantised to multiples of 2^-k (round half to even) and stored
as float32.  With |x| * 2^k < 2^15 every squared distance is an exact FP64
number, which makes the Ball Mapper output a unique, exactly defined object.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

__all__ = [
    "quantise", "isotropic", "mixture", "swissroll", "batched_instances",
    "Workload", "WORKLOADS", "make", "paper_gaussian_fp64", "line_points",
    "grid_points", "tiny_grid_cloud",
]


def quantise(x: np.ndarray, k: int) -> np.ndarray:
    """Round to the nearest multiple of 2^-k (ties to even) and store as float32."""
    scale = float(2 ** k)
    q = np.round(np.asarray(x, dtype=np.float64) * scale) / scale
    out = q.astype(np.float32)
    if not np.array_equal(out.astype(np.float64), q):
        raise ValueError("quantised value not representable in float32")
    return out


def isotropic(n: int, d: int, k: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return quantise(rng.standard_normal((n, d)), k)


def mixture(n: int, d: int, k: int, clusters: int = 32, seed: int = 0,
            half_width: float = 10.0, sigma: float = 1.0) -> np.ndarray:
    """Equal-weight Gaussian mixture; cluster labels are a seeded permutation."""
    if n % clusters:
        raise ValueError("n must be a multiple of the cluster count")
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-half_width, half_width, (clusters, d))
    lab = rng.permutation(np.repeat(np.arange(clusters), n // clusters))
    x = centres[lab] + sigma * rng.standard_normal((n, d))
    return quantise(x, k)


def swissroll(n: int, d: int, k: int, seed: int = 0, noise: float = 0.01) -> np.ndarray:
    rng = np.random.default_rng(seed)
    t = rng.uniform(1.5 * math.pi, 4.5 * math.pi, n)
    h = rng.uniform(0.0, 20.0, n)
    p = np.stack([t * np.cos(t), h, t * np.sin(t)], axis=1)
    frame = np.linalg.qr(rng.standard_normal((d, 3)))[0]          # d x 3, orthonormal columns
    x = p @ frame.T + noise * rng.standard_normal((n, d))
    return quantise(x, k)


@dataclasses.dataclass
class Instance:
    x: np.ndarray
    eps: float
    kind: str


def batched_instances(count: int = 256, k: int = 10, seed: int = 0,
                      n_lo: int = 1000, n_hi: int = 200000,
                      dims: Sequence[int] = (8, 32, 96)) -> List[Instance]:
    """Uneven independent instances: n log-uniform, d from ``dims``, eps U[1, 5]."""
    rng = np.random.default_rng(seed)
    out: List[Instance] = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(rng.choice(np.asarray(dims)))
        kind = int(rng.integers(2))
        eps = float(np.float32(rng.uniform(1.0, 5.0)))
        if kind == 0:
            x = rng.standard_normal((n, d))
        else:
            centres = rng.uniform(-10.0, 10.0, (8, d))
            lab = rng.integers(0, 8, n)
            x = centres[lab] + rng.standard_normal((n, d))
        out.append(Instance(quantise(x, k), eps, "iso" if kind == 0 else "mix8"))
    return out


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    kind: str
    n: int
    d: int
    k: int
    eps: tuple

    def points(self, seed: int = 0) -> np.ndarray:
        if self.kind == "isotropic":
            return isotropic(self.n, self.d, self.k, seed)
        if self.kind == "mixture":
            return mixture(self.n, self.d, self.k, seed=seed)
        if self.kind == "swissroll":
            return swissroll(self.n, self.d, self.k, seed)
        raise ValueError(self.kind)


# The five workload shapes, plus reduced-n variants of the same recipes that
# the oracle finishes in seconds (used as parity cases).
WORKLOADS = {
    "iso-n10k-d16": Workload("iso-n10k-d16", "isotropic", 10_000, 16, 10, (3.0,)),
    "mix32-n1M-d64": Workload("mix32-n1M-d64", "mixture", 1_000_000, 64, 8, (2.0, 4.0, 6.0)),
    "roll-n2M-d128": Workload("roll-n2M-d128", "swissroll", 2_000_000, 128, 12, (0.5, 1.0)),
    "iso-n1M-d128": Workload("iso-n1M-d128", "isotropic", 1_000_000, 128, 10, (14.0,)),
    # reduced variants
    "mix32-n32k-d64": Workload("mix32-n32k-d64", "mixture", 32_768, 64, 8, (2.0, 6.0, 11.0)),
    "roll-n50k-d128": Workload("roll-n50k-d128", "swissroll", 50_000, 128, 12, (0.5, 1.0, 2.0)),
    "iso-n20k-d128": Workload("iso-n20k-d128", "isotropic", 20_000, 128, 10, (14.0,)),
}


def make(name: str, seed: int = 0) -> np.ndarray:
    return WORKLOADS[name].points(seed)


def paper_gaussian_fp64(n: int = 20_000, d: int = 50, seed: int = 0) -> np.ndarray:
    """Unquantised FP64 isotropic Gaussian of the paper's worked example (Sec. 6.3)."""
    return np.random.default_rng(seed).standard_normal((n, d))


def line_points(count: int, d: int = 1) -> np.ndarray:
    """Points i * e_0, i = 0..count-1."""
    x = np.zeros((count, d), dtype=np.float32)
    x[:, 0] = np.arange(count, dtype=np.float32)
    return x


def grid_points(side: int) -> np.ndarray:
    """side x side integer grid in R^2, row-major ids."""
    ii, jj = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    return np.stack([ii.ravel(), jj.ravel()], axis=1).astype(np.float32)


def tiny_grid_cloud(n: int, d: int, k: int, span: int, seed: int) -> np.ndarray:
    """Tiny cloud on the coarse grid (integers in [-span, span]) * 2^-k: many ties."""
    rng = np.random.default_rng(seed)
    m = rng.integers(-span, span + 1, size=(n, d))
    return (m.astype(np.float64) / float(2 ** k)).astype(np.float32)
