"""Batched builds: one bm_build_batched call (the greedy loops of all instances in
one CUDA graph) against one bm_build call per instance, on the same instances.

Both arms run on device-resident inputs; each is timed with CUDA events around
the whole set of instances after warm-up runs, and every instance's result from
the batched arm is checked equal to its single-build result (landmarks,
offsets, ids, edges).  Prints one JSON line.

    python -m paper_2601_01405_gb300.batched_report --count 256 --reps 3
"""
import argparse
import json
import sys
import time


def _same(a, b):
    import torch
    return all(torch.equal(a[k], b[k]) for k in ("landmarks", "offsets", "ids", "edges"))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--n-lo", type=int, default=1000)
    ap.add_argument("--n-hi", type=int, default=200000)
    ap.add_argument("--path", default="auto")
    ap.add_argument("--batch", type=int, default=0, help="largest candidate batch per step (0 = library default)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--tune-batches", action="store_true",
                    help="also time the batched call with per-instance batches from autotune.tune_batches")
    ap.add_argument("--batches-table", default=None, help="a saved autotune --batches table to use instead")
    a = ap.parse_args(argv)

    import torch
    from paper_2601_01405_gb300 import binding, workloads

    t0 = time.perf_counter()
    inst = workloads.batched_instances(count=a.count, seed=a.seed, n_lo=a.n_lo, n_hi=a.n_hi)
    dev = [(torch.from_numpy(i.x).cuda(), i.eps) for i in inst]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0

    def batched():
        return binding.bm_build_batched(dev, path=a.path, batch=a.batch)

    def singles():
        return [binding.bm_build(X, e, path=a.path, batch=a.batch) for X, e in dev]

    def timed(fn):
        ms = []
        out = None
        for r in range(a.warmup + a.reps):
            out = None
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            if r >= a.warmup:
                ms.append(e0.elapsed_time(e1))
        return out, ms

    res_b, ms_b = timed(batched)
    res_s, ms_s = timed(singles)
    mismatches = [k for k, (x, y) in enumerate(zip(res_b, res_s)) if not _same(x, y)]
    tuned = None
    if a.tune_batches or a.batches_table:
        from paper_2601_01405_gb300 import autotune
        t1 = time.perf_counter()
        table = autotune.load(a.batches_table) if a.batches_table else autotune.tune_batches()
        tune_s = time.perf_counter() - t1
        per = autotune.batches_for(table, dev)
        res_t, ms_t = timed(lambda: binding.bm_build_batched(dev, path=a.path, batch=a.batch, batches=per))
        mismatches += [k for k, (x, y) in enumerate(zip(res_t, res_s)) if not _same(x, y)]
        tuned = {"batched_ms": ms_t, "speedup_vs_single": min(ms_s) / min(ms_t),
                 "speedup_vs_untuned": min(ms_b) / min(ms_t), "tune_s": tune_s,
                 "batch_histogram": {str(b): per.count(b) for b in sorted(set(per))},
                 "table": {str(d): [(r["n_lo"], r["n_hi"], r["best"]) for r in rows] for d, rows in table.items()}}
    paths = [int(r["stats"]["path"]) for r in res_b]
    evals = sum(int(r["stats"]["distance_evals"]) for r in res_s)
    L = sum(int(r["landmarks"].numel()) for r in res_s)
    nnz = sum(int(r["ids"].numel()) for r in res_s)
    E = sum(int(r["edges"].shape[0]) for r in res_s)
    launches_b = sum(int(r["stats"]["kernel_launches"]) for r in res_b)
    launches_s = sum(int(r["stats"]["kernel_launches"]) for r in res_s)
    best_b, best_s = min(ms_b), min(ms_s)
    dims = sorted({int(X.shape[1]) for X, _ in dev})
    print(json.dumps({
        "workload": "batched-%d-n%d..%d-d%s" % (a.count, a.n_lo, a.n_hi, "/".join(map(str, dims))),
        "path": a.path, "batch": a.batch,
        "points": int(sum(X.shape[0] for X, _ in dev)), "landmarks": L, "memberships": nnz, "edges": E,
        "distance_evals": evals,
        "batched_ms": ms_b, "single_ms": ms_s,
        "batched_instances_per_s": a.count / (best_b / 1e3), "single_instances_per_s": a.count / (best_s / 1e3),
        "speedup": best_s / best_b,
        "batched_breakdown_ms": ({k: res_b[0]["stats"][k] for k in ("ms_total", "ms_prep", "ms_greedy", "ms_members")}
                                 if res_b else {}),
        "kernels_batched": launches_b, "kernels_single": launches_s,
        "instance_paths": {"split": paths.count(binding.BM_PATH_TC_SPLIT3), "fp16": paths.count(binding.BM_PATH_TC_FP16),
                           "fp32": paths.count(binding.BM_PATH_FP32)},
        "tuned_batches": tuned,
        "mismatched_instances": mismatches, "generate_s": gen_s}))
    return 0 if not mismatches else 1


if __name__ == "__main__":
    sys.exit(main())
