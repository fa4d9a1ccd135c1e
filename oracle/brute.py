"""A second brute-force Ball Mapper, written differently -- TEST INFRASTRUCTURE ONLY.

It pins the C oracle on tiny inputs.  Coordinates must be multiples of 2^-k;
every distance is then compared as an exact rational number:

  D(x, y) < eps^2   <=>   sum_i (m_x,i - m_y,i)^2  <  eps^2 * 4^k

with integer m = x * 2^k and eps^2 * 4^k held as a Fraction.

The greedy, memberships and edges are phrased through sets and witnesses
rather than the C oracle's scans and list intersections:
  * landmarks: repeatedly take min(uncovered), remove its open ball (Sec. 2.2);
  * membership of l: the set comprehension {y : D(l, y) < eps^2} (Sec. 2.3);
  * edge {i, j}: some point x is a witness, D(x,l_i) < eps^2 and
    D(x,l_j) < eps^2 (Sec. 2.1 nerve; equivalently witness radius < eps,
    Sec. 5.2, Def. 5.9).
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations

import numpy as np


def _ints(X, k: int):
    scale = 2 ** k
    out = []
    for row in np.asarray(X, dtype=np.float64):
        r = []
        for v in row:
            f = Fraction(float(v)) * scale
            if f.denominator != 1:
                raise ValueError("coordinate is not a multiple of 2^-k")
            r.append(int(f))
        out.append(tuple(r))
    return out


def build(X, eps, k: int) -> dict:
    pts = _ints(X, k)
    n = len(pts)
    lim = Fraction(float(eps)) ** 2 * (4 ** k)

    def inside(a, b):
        return sum((p - q) ** 2 for p, q in zip(pts[a], pts[b])) < lim

    uncovered = set(range(n))
    landmarks = []
    while uncovered:
        x = min(uncovered)
        landmarks.append(x)
        uncovered -= {y for y in range(n) if inside(x, y)}
    members = [sorted(y for y in range(n) if inside(l, y)) for l in landmarks]
    edge_list = []
    for i, j in combinations(range(len(landmarks)), 2):
        if any(inside(landmarks[i], x) and inside(landmarks[j], x) for x in range(n)):
            edge_list.append((i, j))
    return {"landmarks": landmarks, "members": members, "edges": edge_list}


def fps(X, eps, k: int, first: int = 0) -> list:
    """Farthest point sampling (Sec. 2.2) in exact integer arithmetic: distances to the
    landmark set as exact squared integers, the farthest point (smallest index among
    equal maxima) joins while its squared distance is at least eps^2 * 4^k."""
    pts = _ints(X, k)
    n = len(pts)
    if n == 0:
        return []
    lim = Fraction(float(eps)) ** 2 * (4 ** k)

    def sq(a, b):
        return sum((p - q) ** 2 for p, q in zip(pts[a], pts[b]))

    chosen = [first]
    while True:
        far = {x: min(sq(x, l) for l in chosen) for x in range(n)}
        top = max(far.values())
        if top < lim:
            return chosen
        chosen.append(min(x for x in range(n) if far[x] == top))
