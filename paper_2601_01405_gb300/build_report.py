"""Time whole exact builds (greedy, memberships, nerve edges) on a named workload.

For each eps of the workload (or those given): one warm-up build, then ``reps``
timed builds on device-resident points; prints one JSON line per eps with the
result sizes and the median of the library's phase timings (CUDA events).

    python -m paper_2601_01405_gb300.build_report --workload roll-n2M-d128
"""
import argparse
import json
import statistics
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="roll-n2M-d128")
    ap.add_argument("--eps", type=float, nargs="*", default=None)
    ap.add_argument("--path", choices=["auto", "tc", "tc16", "fp32"], default="auto")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--batch", type=int, default=0, help="largest greedy batch (0 = the library default)")
    ap.add_argument("--skip-edges", action="store_true")
    ap.add_argument("--centring", choices=["auto", "always", "off"], default="auto",
                    help="translation of the tensor-core operands (bm_options.centring)")
    a = ap.parse_args(argv)

    import torch
    from paper_2601_01405_gb300 import binding, workloads

    wl = workloads.WORKLOADS[a.workload]
    X = workloads.make(a.workload)
    Xd = torch.from_numpy(X).cuda()
    for eps in (a.eps or list(wl.eps)):
        binding.bm_build(Xd, eps, path=a.path, batch=a.batch, skip_edges=a.skip_edges, centring=a.centring)
        torch.cuda.synchronize()
        runs = []
        out = None
        for _ in range(a.reps):
            out = None
            out = binding.bm_build(Xd, eps, path=a.path, batch=a.batch, skip_edges=a.skip_edges,
                                   centring=a.centring)
            torch.cuda.synchronize()
            runs.append(out["stats"])
        med = {k: statistics.median(r[k] for r in runs)
               for k in ("ms_total", "ms_prep", "ms_greedy", "ms_members", "ms_edges", "ms_sweep")}
        st = runs[-1]
        print(json.dumps({"workload": a.workload, "eps": eps, "path": a.path, "batch": a.batch, "n": X.shape[0], "d": X.shape[1],
                          "landmarks": int(out["landmarks"].numel()), "memberships": int(out["ids"].numel()),
                          "edges": int(out["edges"].shape[0]), "edge_pairs": st["edge_pairs"],
                          "greedy_steps": st["greedy_steps"], "band_pairs": st["band_pairs"],
                          "band_delta": st["band_delta"], "centring": a.centring, "centred": st["centred"],
                          "path_used": {v: k for k, v in binding.PATHS.items()}.get(st["path"], st["path"]),
                          "distance_evals": st["distance_evals"], "tile_pairs": st["tile_pairs"],
                          "evals_per_s": st["distance_evals"] / (med["ms_total"] / 1e3), "median_ms": med,
                          "tile": binding.get_tile_config(X.shape[1])}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
