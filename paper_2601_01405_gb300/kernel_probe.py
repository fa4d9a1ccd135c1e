"""Run the distance-tile kernel alone on a workload, for profiling and tuning.

One bm_range_query of `rows` query points (the first rows of the point set,
as in one greedy step) against all points of the workload, repeated; prints
the device time of each tile launch.  Example (the shape of one greedy step
on the 1M x 64 mixture):

    python -m paper_2601_01405_gb300.kernel_probe --workload mix32-n1M-d64 --rows 1024 --eps 4 --path tc
"""
import argparse
import json
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="mix32-n1M-d64")
    ap.add_argument("--rows", type=int, default=1024)
    ap.add_argument("--eps", type=float, default=4.0)
    ap.add_argument("--path", choices=["auto", "tc", "tc16", "fp32"], default="auto")
    ap.add_argument("--repeat", type=int, default=3)
    a = ap.parse_args(argv)

    import torch
    from paper_2601_01405_gb300 import binding, workloads

    X = workloads.make(a.workload)
    Xd = torch.from_numpy(X).cuda()
    Qd = Xd[: a.rows].contiguous()
    out = []
    for _ in range(a.repeat):
        off, ids, st = binding.bm_range_query(Xd, Qd, a.eps, path=a.path)
        torch.cuda.synchronize()
        out.append({"ms_sweep": st["ms_sweep"], "ms_total": st["ms_total"], "nnz": int(ids.numel()),
                    "band_pairs": st["band_pairs"], "tile_pairs": st["tile_pairs"]})
    d = X.shape[1]
    best = min(o["ms_sweep"] for o in out)
    pairs = out[0]["tile_pairs"]
    print(json.dumps({"workload": a.workload, "rows": a.rows, "path": a.path, "runs": out,
                      "best_ms_sweep": best, "alg_tflops": 2.0 * d * pairs / (best / 1e3) / 1e12}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
