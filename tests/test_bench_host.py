"""Host-side logic of bench.py on the CPU: the replica aggregation over a gloo
process group of world size 2, and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = [2.0, 3.0][rank]
    evals = [1e12, 3e12][rank]
    rate, smax, esum = bench.aggregate(dist, "cpu", secs, evals)
    with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
        json.dump([rate, smax, esum], f)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_gloo_world2(tmp_path):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        rate, smax, esum = json.load(open(tmp_path / ("r%d.json" % r)))
        assert smax == 3.0 and esum == 4e12
        assert rate == pytest.approx(4e12 / 3.0)


def test_aggregate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(None, "cpu", 2.0, 10.0) == (5.0, 2.0, 10.0)


def test_reference_arm_line():
    """--impl reference times the CPU oracle and prints one JSON line with the contract's keys."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "iso-n10k-d16", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "evals/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_oracle_small_build_timing():
    """The oracle's whole small build with one thread and with all threads, and the
    thread count restored afterwards."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    before = oracle.num_threads()
    out = bench.oracle_small_build()
    assert out["workload"] == "iso-n10k-d16" and out["threads"] == before
    assert out["s_1_thread"] > 0 and out["s_all_threads"] > 0
    assert oracle.num_threads() == before
