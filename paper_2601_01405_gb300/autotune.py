"""Autotuner for the tensor-core distance tiles and the batched greedy's batch sizes.

For each point dimension d it times every compiled tile shape (and each valid
padding of d for it) on the sweep of a greedy step: ``rows`` query rows against
``n`` points with radii so small that almost no pair is a hit, which is the
shape of the greedy's dominant work when most points end up landmarks.  The
fastest configuration per d can be installed in the library
(``bm_set_tile_config``) and saved to / loaded from a JSON file.

Timing is the device time of the tile launches only (the library's sweep
events), the median over ``reps`` calls after one warm-up call.

    python -m paper_2601_01405_gb300.autotune --dims 8 32 64 96 128 --out tiles.json

Greedy batch sizes (``--batches``): for each dimension and range of n of the batched
workload recipe, a set of instances is built with bm_build_batched at every candidate
largest batch (candidates per greedy step), and the fastest is kept; ``batches_for``
then gives every instance of a batched call its tuned batch from that table.

    python -m paper_2601_01405_gb300.autotune --batches --out batches.json
"""
from __future__ import annotations

import argparse
import json
import statistics
import sys
from typing import Dict, Iterable, List


def _paddings(d: int, ck: int) -> List[int]:
    out = {(d + ck - 1) // ck * ck}
    if d > 32:
        out.add((d + 63) // 64 * 64)
    return sorted(p for p in out if p % ck == 0 and p >= d)


def candidates(d: int) -> List[dict]:
    """Every (d_pad, shape) the library accepts for dimension d.  Probing leaves d on
    the built-in choice (any override for d is removed)."""
    from . import binding
    found = []
    for shp in binding.tile_shapes():
        for d_pad in _paddings(d, shp["ck"]):
            cfg = dict(shp, d_pad=d_pad)
            try:
                binding.set_tile_config(d, cfg)
            except binding.BallMapperError:
                continue
            finally:
                binding.set_tile_config(d, None)
            found.append(cfg)
    return found


def time_config(d: int, cfg: dict, X, Q, eps: float, reps: int, path: str = "tc") -> float:
    """Median device time (ms) of the tile launches of one range query under cfg (d is
    left on the built-in choice afterwards)."""
    from . import binding
    import torch
    binding.set_tile_config(d, cfg)
    try:
        binding.bm_range_query(X, Q, eps, path=path)
        ms = []
        for _ in range(reps):
            _, _, st = binding.bm_range_query(X, Q, eps, path=path)
            torch.cuda.synchronize()
            ms.append(st["ms_sweep"])
        return statistics.median(ms)
    finally:
        binding.set_tile_config(d, None)


def tune(dims: Iterable[int], n: int = 200_000, rows: int = 2048, reps: int = 5, seed: int = 0,
         path: str = "tc") -> Dict[int, dict]:
    """{d: {"best": cfg, "builtin": cfg, "timings": [(cfg, ms), ...]}}."""
    import torch
    from . import binding, workloads
    out = {}
    for d in dims:
        X = torch.from_numpy(workloads.isotropic(n, d, 10, seed=seed + d)).cuda()
        Q = X[:rows].contiguous()
        eps = 1e-3  # only the self pairs are hits
        builtin = binding.get_tile_config(d)
        timings = []
        for cfg in candidates(d):
            timings.append((cfg, time_config(d, cfg, X, Q, eps, reps, path)))
        timings.sort(key=lambda t: t[1])
        out[d] = {"path": path, "best": timings[0][0], "best_ms": timings[0][1], "builtin": builtin,
                  "builtin_ms": next((ms for c, ms in timings if c == builtin), None),
                  "evals": n * rows, "timings": [{"cfg": c, "ms": ms} for c, ms in timings]}
    return out


BATCH_CHOICES = (128, 256, 512, 1024, 2048)
N_BUCKETS = ((1000, 5000), (5000, 30000), (30000, 200000))


def tune_batches(dims: Iterable[int] = (8, 32, 96), buckets=N_BUCKETS, count: int = 12,
                 choices=BATCH_CHOICES, reps: int = 3, seed: int = 0) -> Dict[int, list]:
    """{d: [{"n_lo", "n_hi", "best", "ms": {batch: ms}}, ...]}: per dimension and range of n,
    the largest greedy batch with the shortest bm_build_batched time (CUDA events, median of
    reps after one warm-up) on `count` instances of the batched recipe in that range."""
    import torch
    from . import binding, workloads
    out: Dict[int, list] = {}
    for d in dims:
        rows = []
        for lo, hi in buckets:
            inst = workloads.batched_instances(count=count, seed=seed + 7 * d + lo, n_lo=lo, n_hi=hi, dims=(d,))
            dev = [(torch.from_numpy(i.x).cuda(), i.eps) for i in inst]
            ms = {}
            for b in choices:
                binding.bm_build_batched(dev, batch=b)
                torch.cuda.synchronize()
                t = []
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    binding.bm_build_batched(dev, batch=b)
                    e1.record()
                    torch.cuda.synchronize()
                    t.append(e0.elapsed_time(e1))
                ms[b] = statistics.median(t)
            rows.append({"n_lo": lo, "n_hi": hi, "best": min(ms, key=ms.get), "ms": ms})
        out[d] = rows
    return out


def batches_for(table: Dict, instances) -> List[int]:
    """Per-instance largest batch from a tune_batches table: the entry of the nearest tuned
    dimension whose range of n holds the instance (the nearest range otherwise)."""
    dims = sorted(int(k) for k in table)
    res = []
    for X, _ in instances:
        n, d = int(X.shape[0]), int(X.shape[1])
        dd = min(dims, key=lambda v: (abs(v - d), v))
        rows = table[dd] if dd in table else table[str(dd)]
        row = min(rows, key=lambda r: 0 if r["n_lo"] <= n < r["n_hi"] else min(abs(n - r["n_lo"]), abs(n - r["n_hi"])))
        res.append(int(row["best"]))
    return res


def install(table: Dict) -> None:
    """Install the best configuration of each d of a tune() result or saved file."""
    from . import binding
    for d, entry in table.items():
        binding.set_tile_config(int(d), entry["best"])


def save(table: Dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump({str(d): v for d, v in table.items()}, f, indent=1)


def load(path: str) -> Dict[int, dict]:
    with open(path) as f:
        return {int(d): v for d, v in json.load(f).items()}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs="+", default=[8, 32, 64, 96, 128])
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--rows", type=int, default=2048)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--out", default=None)
    ap.add_argument("--path", choices=["tc", "tc16"], default="tc", help="tensor-core representation to time")
    ap.add_argument("--batches", action="store_true", help="tune the batched greedy's batch sizes instead")
    a = ap.parse_args(argv)
    if a.batches:
        table = tune_batches(a.dims if a.dims != [8, 32, 64, 96, 128] else (8, 32, 96), reps=a.reps)
        if a.out:
            with open(a.out, "w") as f:
                json.dump({str(d): v for d, v in table.items()}, f, indent=1)
        for d, rows in table.items():
            print(json.dumps({"d": d, "rows": rows}))
        return 0
    table = tune(a.dims, a.n, a.rows, a.reps, path=a.path)
    if a.out:
        save(table, a.out)
    for d, e in table.items():
        rate = lambda ms: e["evals"] / (ms * 1e-3) if ms else None
        print(json.dumps({"d": d, "best": e["best"], "best_evals_per_s": rate(e["best_ms"]), "builtin": e["builtin"],
                          "builtin_evals_per_s": rate(e["builtin_ms"]),
                          "all": [(t["cfg"]["d_pad"], t["cfg"]["ck"], t["cfg"]["nt"], t["cfg"]["bbuf"],
                                   t["cfg"]["astg"], round(t["ms"], 4)) for t in e["timings"]]}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
