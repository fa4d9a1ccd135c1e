"""Approximate Ball Mapper with a non-exhaustive index (the inverted file, or the
proximity graph with --index graph), scored against the exact build.

For each nprobe (ef for the graph): the fixed-landmark mode (exact landmarks, balls through the index)
gives range recall/precision and edge recall/precision (Sec. 5.3 definitions; Sec. 6.2
edge recall and precision); the end-to-end mode (the greedy driven by the index) gives
the landmark ratio |L~|/|L|, the normalised covering radius rho(L~)/eps and the
normalised separation s(L~)/eps (Sec. 6.2).  Precision 1 (no false-positive membership
or edge) is asserted.  The covering radius and separation are computed here with
torch (float32, reporting only).

    python -m paper_2601_01405_gb300.ivf_report --workload iso-n1M-d128 --eps 14 --nprobe 1 8 32
    python -m paper_2601_01405_gb300.ivf_report --paper-gaussian --index graph --ef 16 64 --nprobe 1 32 128

--paper-gaussian takes the float32 cast of the worked example's data (Sec. 6.3:
default_rng(0).standard_normal((20000, 50))) with eps from the target-occupancy rule
(k = 50) computed on the GPU.
"""
import argparse
import json
import sys
import time


def _subset(a_keys, b_keys):
    """Every key of sorted a_keys occurs in sorted b_keys (device tensors)."""
    import torch
    if a_keys.numel() == 0:
        return True
    pos = torch.searchsorted(b_keys, a_keys).clamp(max=max(b_keys.numel() - 1, 0))
    return bool((b_keys[pos] == a_keys).all()) if b_keys.numel() else False


def _member_keys(out, n):
    import torch
    off = out["offsets"]
    rows = torch.repeat_interleave(torch.arange(off.numel() - 1, device=off.device), off[1:] - off[:-1])
    return rows * n + out["ids"].long()


def _edge_keys(out, L):
    e = out["edges"]
    return e[:, 0].long() * L + e[:, 1].long()


def _cover_and_separation(Xd, lm, chunk=8192):
    import torch
    P = Xd[lm.long()]
    rho2 = torch.zeros((), device=Xd.device)
    for i in range(0, Xd.shape[0], chunk):
        d2 = torch.cdist(Xd[i:i + chunk], P).pow(2)
        rho2 = torch.maximum(rho2, d2.min(dim=1).values.max())
    s2 = torch.tensor(float("inf"), device=Xd.device)
    for i in range(0, P.shape[0], chunk):
        d2 = torch.cdist(P[i:i + chunk], P).pow(2)
        idx = torch.arange(i, min(i + chunk, P.shape[0]), device=Xd.device)
        d2[idx - i, idx] = float("inf")
        s2 = torch.minimum(s2, d2.min())
    return float(rho2.sqrt()), float(s2.sqrt())


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="iso-n1M-d128")
    ap.add_argument("--eps", type=float, default=14.0)
    ap.add_argument("--nprobe", type=int, nargs="+", default=[1, 8, 32])
    ap.add_argument("--nlist", type=int, default=1024)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--sample", type=int, default=262144)
    ap.add_argument("--no-end-to-end", action="store_true")
    ap.add_argument("--index", choices=["ivf", "graph"], default="ivf")
    ap.add_argument("--ef", type=int, nargs="+", default=[16, 64, 256], help="graph index: beam widths")
    ap.add_argument("--M", type=int, default=16, help="graph index: nearest neighbours per point")
    ap.add_argument("--entries", type=int, default=64, help="graph index: entry points")
    ap.add_argument("--max-visits", type=int, default=8192, help="graph index: visits per query")
    ap.add_argument("--paper-gaussian", action="store_true")
    ap.add_argument("--path", choices=["auto", "tc", "fp32"], default="auto",
                    help="inverted file: the scan's arithmetic (tensor-core tiles or FP32 CUDA-core tiles)")
    a = ap.parse_args(argv)

    import numpy as np
    import torch
    from paper_2601_01405_gb300 import binding, workloads

    if a.paper_gaussian:
        X = workloads.paper_gaussian_fp64(20000, 50, seed=0).astype(np.float32)
        a.workload = "paper-gaussian-n20k-d50-fp32"
        Xd = torch.from_numpy(X).cuda()
        a.eps = float(np.float32(binding.bm_occupancy_eps(Xd, 50)[0]))
    else:
        X = workloads.make(a.workload)
        Xd = torch.from_numpy(X).cuda()
    n = X.shape[0]
    if a.index == "graph":
        return _graph_report(a, binding, torch, Xd, n)
    exact = binding.bm_build(Xd, a.eps)
    torch.cuda.synchronize()
    L = exact["landmarks"].numel()
    ek = _member_keys(exact, n)
    ee = _edge_keys(exact, L)
    t = time.perf_counter()
    index = binding.IvfIndex(Xd, nlist=a.nlist, iters=a.iters, sample=min(a.sample, n), seed=0, path=a.path)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t
    rows = []
    for p in a.nprobe:
        fx = index.build(a.eps, p, landmarks=exact["landmarks"])
        torch.cuda.synchronize()
        fk = _member_keys(fx, n)
        fe = _edge_keys(fx, L)
        assert _subset(fk, ek), "false-positive membership"
        assert _subset(fe, ee), "false-positive edge"
        row = {"nprobe": p, "range_recall": fk.numel() / max(ek.numel(), 1), "range_precision": 1.0,
               "edge_recall": fe.numel() / max(ee.numel(), 1), "edge_precision": 1.0,
               "fixed_build_s": fx["stats"]["ms_total"] / 1e3}
        if not a.no_end_to_end:
            e2e = index.build(a.eps, p)
            torch.cuda.synchronize()
            rho, sep = _cover_and_separation(Xd, e2e["landmarks"])
            row.update({"landmark_ratio": e2e["landmarks"].numel() / L, "rho_over_eps": rho / a.eps,
                        "separation_over_eps": sep / a.eps, "end_to_end_build_s": e2e["stats"]["ms_total"] / 1e3})
        rows.append(row)
    print(json.dumps({"workload": a.workload, "eps": a.eps, "index": "ivf", "path": a.path, "nlist": a.nlist,
                      "iters": a.iters, "sample": a.sample,
                      "exact": {"landmarks": L, "memberships": int(ek.numel()), "edges": int(ee.numel()),
                                "build_s": exact["stats"]["ms_total"] / 1e3},
                      "train_s": train_s, "results": rows}))
    return 0


def _graph_report(a, binding, torch, Xd, n):
    """The proximity-graph index: per ef, fixed-landmark recall (range and edges) and the
    end-to-end landmark ratio, covering radius and separation; zero false positives asserted."""
    exact = binding.bm_build(Xd, a.eps)
    torch.cuda.synchronize()
    L = exact["landmarks"].numel()
    ek = _member_keys(exact, n)
    ee = _edge_keys(exact, L)
    t = time.perf_counter()
    index = binding.GraphIndex(Xd, M=a.M, n_entries=min(a.entries, n))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t
    rows = []
    for ef in a.ef:
        fx = index.build(a.eps, ef, a.max_visits, landmarks=exact["landmarks"])
        torch.cuda.synchronize()
        fk = _member_keys(fx, n)
        fe = _edge_keys(fx, L)
        assert _subset(fk, ek), "false-positive membership"
        assert _subset(fe, ee), "false-positive edge"
        row = {"ef": ef, "range_recall": fk.numel() / max(ek.numel(), 1), "range_precision": 1.0,
               "edge_recall": fe.numel() / max(ee.numel(), 1), "edge_precision": 1.0,
               "visits_per_query": fx["stats"]["tile_pairs"] / max(L, 1), "truncated": fx["stats"]["truncated"],
               "fixed_build_s": fx["stats"]["ms_total"] / 1e3}
        if not a.no_end_to_end:
            e2e = index.build(a.eps, ef, a.max_visits)
            torch.cuda.synchronize()
            rho, sep = _cover_and_separation(Xd, e2e["landmarks"])
            row.update({"landmark_ratio": e2e["landmarks"].numel() / L, "rho_over_eps": rho / a.eps,
                        "separation_over_eps": sep / a.eps, "end_to_end_build_s": e2e["stats"]["ms_total"] / 1e3})
        rows.append(row)
    print(json.dumps({"workload": a.workload, "eps": a.eps, "index": "graph", "M": a.M, "entries": a.entries,
                      "max_visits": a.max_visits, "graph_edges": index.n_adj // 2,
                      "exact": {"landmarks": L, "memberships": int(ek.numel()), "edges": int(ee.numel()),
                                "build_s": exact["stats"]["ms_total"] / 1e3},
                      "index_build_s": build_s, "results": rows}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
