"""Approximate Ball Mapper with the inverted-file index, scored against the exact build.

For each nprobe: the fixed-landmark mode (exact landmarks, balls through the index)
gives range recall/precision and edge recall/precision (Sec. 5.3 definitions; Sec. 6.2
edge recall and precision); the end-to-end mode (the greedy driven by the index) gives
the landmark ratio |L~|/|L|, the normalised covering radius rho(L~)/eps and the
normalised separation s(L~)/eps (Sec. 6.2).  Precision 1 (no false-positive membership
or edge) is asserted.  The covering radius and separation are computed here with
torch (float32, reporting only).

    python -m paper_2601_01405_gb300.ivf_report --workload iso-n1M-d128 --eps 14 --nprobe 1 8 32
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
    a = ap.parse_args(argv)

    import torch
    from paper_2601_01405_gb300 import binding, workloads

    X = workloads.make(a.workload)
    Xd = torch.from_numpy(X).cuda()
    n = X.shape[0]
    exact = binding.bm_build(Xd, a.eps)
    torch.cuda.synchronize()
    L = exact["landmarks"].numel()
    ek = _member_keys(exact, n)
    ee = _edge_keys(exact, L)
    t = time.perf_counter()
    index = binding.IvfIndex(Xd, nlist=a.nlist, iters=a.iters, sample=min(a.sample, n), seed=0)
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
    print(json.dumps({"workload": a.workload, "eps": a.eps, "nlist": a.nlist, "iters": a.iters, "sample": a.sample,
                      "exact": {"landmarks": L, "memberships": int(ek.numel()), "edges": int(ee.numel()),
                                "build_s": exact["stats"]["ms_total"] / 1e3},
                      "train_s": train_s, "results": rows}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
