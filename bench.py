#!/usr/bin/env python
"""Benchmark: exact Ball Mapper construction on one GB300 (or N independent replicas).

Workload (default): equal-weight 32-cluster Gaussian mixture, n = 1,000,000 points,
d = 64, centres U[-10,10]^64, sigma = 1, coordinates quantised to multiples of 2^-8
and stored as float32, eps in {2, 4, 6}, greedy in index order.  One step = one
complete bm_build (prep, block-greedy with full-ball memberships, CSR, nerve edges)
for each of the three eps values, inputs resident in HBM.

Metric: exact distance evaluations per second, where one evaluation is one
(landmark, point) membership decision: sum over eps of L_eps * n per step.
The build seconds per eps, the plain FP32 CUDA-core path on the same workload,
the roofline of the tensor-core distance tiles and the CPU oracle are reported
beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Kernel-only mode, for profiling one distance-tile launch shape: one bm_range_query
of the first ROWS points (the shape of one greedy step) against all points of the
workload, repeated, printing the device time of the tile launches:

  python bench.py --kernel-probe --workload mix32-n1M-d64 --rows 8192 --eps 4 --path tc16
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Ball Mapper build s & distance evals/s (exact), TC split path vs plain FP32"
UNIT = "evals/s"
# DRAM bytes per tile-kernel launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# an ncu capture of the current fp16 kernel at the greedy's full batch (16384 candidate
# rows x 10^6 points); a step's sweep reads every point's operands once whatever its
# batch, so the figure holds for each launch of this workload to within the query rows'
# 160 B each (the automatic path runs fp16 after the first step).  None where no capture
# of the current kernel exists.
NCU_TRAFFIC = {("mix32-n1M-d64", "auto"): 166.5e6, ("mix32-n1M-d64", "tc16"): 166.5e6}
DTYPES = {"tc": "bf16x3-split/fp32-acc/fp64-recheck", "tc16": "f16-scaled/fp32-acc/fp64-recheck",
          "fp32": "f32/fp64-recheck", "auto": "f16-scaled or bf16x3-split/fp32-acc/fp64-recheck"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="mix32-n1M-d64")
    ap.add_argument("--path", choices=["auto", "tc", "tc16", "fp32"], default="auto")
    ap.add_argument("--compare-steps", type=int, default=1, help="timed steps of the FP32 comparison path (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline sample")
    ap.add_argument("--dists-builds", type=int, default=1,
                    help="untimed builds per eps with reported distances (their measured error); 0: skip")
    ap.add_argument("--other-configs", type=int, default=1,
                    help="also time whole builds of the other configurations (1 rank, N = 1 only; 0: skip)")
    ap.add_argument("--kernel-probe", action="store_true",
                    help="time one distance-tile launch shape (a range query of --rows rows) and exit")
    ap.add_argument("--rows", type=int, default=1024, help="query rows of the kernel probe")
    ap.add_argument("--eps", type=float, default=4.0, help="eps of the kernel probe")
    ap.add_argument("--repeat", type=int, default=3, help="repetitions of the kernel probe")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(name):
    from paper_2601_01405_gb300 import workloads as W
    w = W.WORKLOADS[name]
    return w, w.points(0)


def config_of(w, extra=None):
    cfg = {"workload": "%s: %s n=%d d=%d quantised 2^-%d, eps=%s, greedy in index order" %
                       (w.name, w.kind, w.n, w.d, w.k, list(w.eps)),
           "n": w.n, "d": w.d, "eps": list(w.eps), "quantisation": "2^-%d" % w.k,
           "l2": "inputs larger than L2 (%.0f MB fp32 points; tile operands %.0f MB fp16 or %.0f MB bf16 split; "
                 "L2 129 MB)" % (w.n * w.d * 4 / 1e6, w.n * ((w.d if w.d > 32 else 32) + 16) * 2 / 1e6,
                                 w.n * (2 * (w.d if w.d > 32 else 32) + 16) * 2 / 1e6),
           "parallelism": "replicas"}
    if extra:
        cfg.update(extra)
    return cfg


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def aggregate(dist, device, seconds, evals):
    """Whole-job rate over replicas: evaluations summed over ranks divided by the
    slowest rank's time (max over ranks).  Returns (rate, seconds_max, evals_sum)."""
    if dist is None:
        return evals / seconds, seconds, evals
    import torch
    t_max = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    e_sum = torch.tensor([float(evals)], dtype=torch.float64, device=device)
    dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    dist.all_reduce(e_sum, op=dist.ReduceOp.SUM)
    return float(e_sum.item()) / float(t_max.item()), float(t_max.item()), float(e_sum.item())


# --------------------------------------------------------------------------- CPU oracle
def oracle_rate(X, eps_list, target_s, landmark_rows=None):
    """Time the CPU oracle's full-scan membership query (the same exact decision per
    (row, point) pair as the GPU sweep) on a bounded sample of rows.  Returns
    (evals/s, evals, seconds, rows, threads)."""
    import numpy as np
    import oracle
    n = X.shape[0]
    rng = np.random.default_rng(1)
    # calibration on a few rows, then size the sample to ~target_s
    rows0 = 8
    oracle.range_query(X, X[rng.integers(0, n, 2)], eps_list[0])     # load / first-touch, untimed
    t0 = time.perf_counter()
    oracle.range_query(X, X[rng.integers(0, n, rows0)], eps_list[0])
    dt0 = max(time.perf_counter() - t0, 1e-3)
    rows = max(len(eps_list), int(rows0 * target_s / dt0))
    per = max(1, rows // len(eps_list))
    evals = 0
    t0 = time.perf_counter()
    for e in eps_list:
        q = X[rng.integers(0, n, per)] if landmark_rows is None else X[landmark_rows[:per]]
        oracle.range_query(X, q, e)
        evals += per * n
    dt = time.perf_counter() - t0
    return evals / dt, evals, dt, per * len(eps_list), oracle.num_threads()


def _guarded(fn):
    """A supplementary CPU figure must never cost the benchmark its line."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001
        return {"error": "%s: %s" % (type(e).__name__, e)}


def oracle_small_build(name="iso-n10k-d16", eps=3.0):
    """Whole oracle build (greedy, memberships, edges) of the small configuration with one
    thread and with all threads: the oracle's own scaling, reported beside the sample rate."""
    import oracle
    from paper_2601_01405_gb300 import workloads as W
    X = W.make(name)
    threads = oracle.num_threads()
    oracle.build(X, eps)   # first touch, untimed
    out = {"workload": name, "eps": eps, "threads": threads}
    try:
        for key, th in (("s_1_thread", 1), ("s_all_threads", threads)):
            oracle.set_num_threads(th)
            t0 = time.perf_counter()
            oracle.build(X, eps)
            out[key] = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(threads)
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w, X = workload(args.workload)
    eps_list = list(w.eps)
    step_target = 6.0
    import oracle
    # warm-up steps (untimed) then K timed steps, each a bounded sample of the workload
    rates = []
    t_steps = []
    evals_total = 0
    for i in range(args.warmup + args.steps):
        r, ev, dt, rows, thr = oracle_rate(X, eps_list, step_target)
        if i >= args.warmup:
            rates.append(r)
            t_steps.append(dt)
            evals_total += ev
    value = evals_total / sum(t_steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(t_steps) / len(t_steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": "per step ~%d random query rows x all %d points (full-scan FP64 "
                                       "membership), split over eps %s" % (rows, w.n, eps_list)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch
    from paper_2601_01405_gb300 import binding, _build

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}), flush=True)
        return 1
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    _build.build()
    binding.load()
    w, X = workload(args.workload)
    eps_list = list(w.eps)
    Xd = torch.from_numpy(X).cuda()
    n, d = X.shape
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    def step(path):
        stats = []
        for e in eps_list:
            out = binding.bm_build(Xd, e, path=path)
            stats.append(out["stats"])
            del out
        return stats

    def timed(path, warm, steps):
        for _ in range(warm):
            step(path)
        barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        all_stats = []
        for _ in range(steps):
            all_stats.append(step(path))
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = ev0.elapsed_time(ev1)
        return ms, all_stats

    sampler = ClockSampler(local)
    for _ in range(args.warmup):
        step(args.path)
    sampler.start()
    ms, stats = timed(args.path, 0, args.steps)
    clocks = sampler.stop()
    evals_per_step = sum(s["distance_evals"] for s in stats[0])
    value, secs, _ = aggregate(dist, "cuda", ms / 1000.0, evals_per_step * args.steps)
    ms = secs * 1000.0
    ms_step = ms / args.steps
    flat = [s for st in stats for s in st]
    build_s = {str(e): sum(st[i]["ms_total"] for st in stats) / len(stats) / 1000.0 for i, e in enumerate(eps_list)}
    L_per_eps = {str(e): stats[0][i]["distance_evals"] // n for i, e in enumerate(eps_list)}
    launches = sum(s["kernel_launches"] for s in flat)

    # roofline of the dominant kernel: the tensor-core distance tiles
    pk, pk_kind = peaks()
    sweep_ms = sum(s["ms_sweep"] for s in flat)
    sweep_n = sum(s["sweep_launches"] for s in flat)
    tile_pairs = sum(s["tile_pairs"] for s in flat)
    d_pad = binding.get_tile_config(d)["d_pad"]
    alg_flops = 2.0 * d * tile_pairs
    # tensor-core products per coordinate: three for the bf16 split, one for fp16 (the
    # path each build finished on; the automatic path reports it per build)
    issued_flops = sum(2.0 * ((1 if s["path"] == binding.BM_PATH_TC_FP16 else 3) * d_pad + 16) * s["tile_pairs"]
                       for s in flat)
    achieved = alg_flops / (sweep_ms / 1000.0) / 1e12 if sweep_ms > 0 else 0.0
    peak = pk.get("bf16_tflops_sustained", 1700.0)
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None,
                "traffic": NCU_TRAFFIC.get((args.workload, args.path)),
                "kernel": "sweep_fp32_kernel" if args.path == "fp32" else "sweep_tc_kernel",
                "peak_kind": "%s bf16 sustained" % pk_kind,
                "issued_tflops": issued_flops / (sweep_ms / 1000.0) / 1e12 if sweep_ms > 0 else 0.0,
                "issued_frac": (issued_flops / (sweep_ms / 1000.0) / 1e12) / peak if sweep_ms > 0 and peak else None,
                "avg_launch_ms": sweep_ms / sweep_n if sweep_n else None, "launches": sweep_n,
                "sweep_share_of_step": sweep_ms / ms if ms else None}

    # arithmetic actually used (the automatic path reports the path each build finished on)
    used = sorted({s["path"] for s in flat})
    by_code = {binding.BM_PATH_TC_SPLIT3: "tc", binding.BM_PATH_TC_FP16: "tc16", binding.BM_PATH_FP32: "fp32"}
    dtype_used = " + ".join(DTYPES[by_code[u]] for u in used if u in by_code) or DTYPES[args.path]

    extra = {}
    # comparisons on the same workload: the bf16 hi/lo split tensor-core path (the metric's
    # "TC split path") and the plain FP32 CUDA-core path
    if args.compare_steps > 0:
        for cmp_path, key in (("tc", "split_path"), ("fp32", "fp32_path")):
            if cmp_path == args.path:
                continue
            msc, stc = timed(cmp_path, 1, args.compare_steps)
            evc = sum(s["distance_evals"] for s in stc[0])
            fc = [s for st in stc for s in st]
            extra[key] = {"value": evc * args.compare_steps / (msc / 1000.0), "unit": UNIT,
                          "ms_per_step": msc / args.compare_steps, "steps": args.compare_steps,
                          "build_s": {str(e): fc[i]["ms_total"] / 1000.0 for i, e in enumerate(eps_list)},
                          "band_pairs": sum(s["band_pairs"] for s in fc),
                          "recheck_rate": sum(s["band_pairs"] for s in fc) / max(sum(s["tile_pairs"] for s in fc), 1)}
            if cmp_path == "fp32":
                extra["tc_speedup_vs_fp32"] = (msc / args.compare_steps) / ms_step
                if "split_path" in extra:
                    extra["split_speedup_vs_fp32"] = msc / extra["split_path"]["ms_per_step"] / args.compare_steps
    # reported distances (opt-in output): one untimed build per eps with distances, their
    # measured error against the FP64 distance the oracle computes
    dist_err = []
    for _ in range(args.dists_builds):
        for e in eps_list:
            out = binding.bm_build(Xd, e, path=args.path, want_dists=True)
            dist_err.append(out["stats"]["dist_max_rel_err"])
            del out
    if dist_err:
        extra["dists"] = {"max_rel_err_vs_fp64": max(dist_err), "tolerance": 1e-6,
                          "note": "untimed builds with want_dists, %d per eps" % args.dists_builds}

    # end to end through the C-ABI with host buffers: H2D of the inputs and D2H of the graph inside
    e2e = None
    if args.e2e_steps > 0:
        Xp = torch.from_numpy(X).pin_memory().numpy()
        binding.bm_build(Xp, eps_list[0], path=args.path)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.e2e_steps):
            for e in eps_list:
                out = binding.bm_build(Xp, e, path=args.path)
                L, nnz, E = out["landmarks"].size, out["ids"].size, out["edges"].shape[0]
                d2h += 4 * L + 8 * (L + 1) + 4 * nnz + 8 * E
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e_rate, _, _ = aggregate(dist, "cuda", dt, evals_per_step * args.e2e_steps)
        e2e = {"value": e2e_rate, "unit": UNIT,
               "h2d_bytes_per_step": int(n * d * 4 * len(eps_list)),
               "d2h_bytes_per_step": int(d2h // args.e2e_steps)}

    if rank == 0 and ws == 1 and args.other_configs > 0 and args.workload == "mix32-n1M-d64":
        extra["other_configs"] = _guarded(lambda: other_configs(args.path))

    cpu = None
    if rank == 0 and ws == 1 and args.cpu_seconds > 0:
        r, ev, dt, rows, thr = oracle_rate(X, eps_list, args.cpu_seconds)
        cpu = {"value": r, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": "%d random query rows x all %d points, full-scan FP64 membership, split over eps %s "
                         "(%.1f s)" % (rows, n, eps_list, dt),
               "small_build": _guarded(oracle_small_build)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_used,
            "data": "synthetic (seeded generator, same recipe and sizes as the workload)",
            "config": config_of(w, {"path": args.path, "landmarks": L_per_eps, "build_s": build_s,
                                    "evals_per_step": evals_per_step,
                                    "band_pairs": sum(s["band_pairs"] for s in flat),
                                    "tile_pairs": tile_pairs,
                                    "recheck_rate": sum(s["band_pairs"] for s in flat) / max(tile_pairs, 1)}),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches}
    line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def other_configs(path, reps=3):
    """Whole builds of the other configurations, device-resident inputs: the median of the
    library's CUDA-event total over reps builds after one warm-up, with the result sizes;
    batched-256: the whole bm_build_batched call (CUDA events)."""
    import statistics
    import torch
    from paper_2601_01405_gb300 import binding, workloads as W
    out = []
    for name in ("iso-n10k-d16", "roll-n2M-d128", "iso-n1M-d128"):
        wl = W.WORKLOADS[name]
        Xd = torch.from_numpy(W.make(name)).cuda()
        for e in wl.eps:
            binding.bm_build(Xd, e, path=path)
            runs, g = [], None
            for _ in range(reps):
                g = binding.bm_build(Xd, e, path=path)
                runs.append(g["stats"]["ms_total"])
            out.append({"workload": name, "eps": e, "build_s": statistics.median(runs) / 1e3,
                        "landmarks": int(g["landmarks"].numel()), "memberships": int(g["ids"].numel()),
                        "edges": int(g["edges"].shape[0]),
                        "path_used": {v: k for k, v in binding.PATHS.items()}.get(g["stats"]["path"])})
            del g
        del Xd
    inst = W.batched_instances(count=256)
    dev = [(torch.from_numpy(i.x).cuda(), i.eps) for i in inst]
    binding.bm_build_batched(dev, path=path)
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = binding.bm_build_batched(dev, path=path)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    out.append({"workload": "batched-256", "instances": len(inst), "build_s": statistics.median(ms) / 1e3,
                "landmarks": int(sum(r["landmarks"].numel() for r in res)),
                "memberships": int(sum(r["ids"].numel() for r in res))})
    return out


def run_kernel_probe(args):
    """One range query of the first `rows` points against all points of the workload,
    repeated: the distance-tile launch of one greedy step, alone (for ncu)."""
    import torch
    from paper_2601_01405_gb300 import binding, _build
    _build.build()
    w, X = workload(args.workload)
    Xd = torch.from_numpy(X).cuda()
    Qd = Xd[: args.rows].contiguous()
    runs = []
    for _ in range(args.repeat):
        off, ids, st = binding.bm_range_query(Xd, Qd, args.eps, path=args.path)
        torch.cuda.synchronize()
        runs.append({"ms_sweep": st["ms_sweep"], "ms_total": st["ms_total"], "nnz": int(ids.numel()),
                     "band_pairs": st["band_pairs"], "tile_pairs": st["tile_pairs"]})
    best = min(r["ms_sweep"] for r in runs)
    pairs = runs[0]["tile_pairs"]
    print(json.dumps({"workload": args.workload, "rows": args.rows, "eps": args.eps, "path": args.path,
                      "runs": runs, "best_ms_sweep": best,
                      "alg_tflops": 2.0 * X.shape[1] * pairs / (best / 1e3) / 1e12 if best > 0 else None}))
    return 0


def main():
    args = parse()
    if args.kernel_probe:
        return run_kernel_probe(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
