"""CPU tests of bench.py's multi-rank logic with the gloo backend and two
ranks: the step time is the maximum over ranks, and the reference arm runs
on rank 0 only (the other ranks exit 0 without output)."""
import json
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        q.put((rank, bench.dist_max(10.0 + 5.0 * rank, ws, device="cpu")))
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_dist_max_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 15.0), (1, 15.0)]


def test_dist_max_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_max(3.5, 1) == 3.5


def test_reference_arm_two_ranks():
    """torchrun with two ranks: rank 0 prints the oracle's line, rank 1 exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["e2e"]["h2d_bytes_per_step"] == 0


def test_median_ci95_order_statistics():
    """The step-sample interval: median of the samples and the order
    statistics at ranks n/2 -+ 1.96 sqrt(n)/2; for 40 samples ranks 13 and 27
    (1-based). Coverage of the true median checked on seeded samples."""
    import random
    sys.path.insert(0, ROOT)
    import bench
    med, lo, hi = bench.median_ci95(list(range(40, 0, -1)))  # 1..40 reversed
    assert med == 20.5 and lo == 13 and hi == 27
    med, lo, hi = bench.median_ci95([5.0])
    assert med == lo == hi == 5.0
    rng = random.Random(3)
    hits = 0
    for _ in range(2000):
        xs = [rng.expovariate(1.0) for _ in range(40)]
        _, a, b = bench.median_ci95(xs)
        hits += a <= 0.6931471805599453 <= b  # median of Exp(1) = ln 2
    assert 0.93 <= hits / 2000 <= 0.99


def test_record_traffic_from_ncu_csv_and_hash_check(tmp_path):
    """The traffic recorder averages dram read + write over the kernel's
    launches in an ncu raw CSV (units row honoured), scales it, and the bench
    drops the figure once the recorded source hash no longer matches."""
    import json
    bench = _bench()
    csv = tmp_path / "raw.csv"
    csv.write_text(
        '"ID","Kernel Name","dram__bytes_read.sum","dram__bytes_write.sum"\n'
        '"","","Mbyte","Kbyte"\n'
        '"0","void k_stencil_tma<double>(...)","100.5","2,000"\n'
        '"1","k_fixup_f64(...)","7","7"\n'
        '"2","void k_stencil_tma<double>(...)","99.5","2,000"\n')
    out = tmp_path / "traffic.json"
    rec = bench.record_traffic(str(csv), "k", "k_stencil_tma", 8.0, "test", path=str(out))
    assert rec["launches"] == 2
    assert rec["captured_bytes_per_launch"] == int(100e6 + 2e6)
    assert rec["dram_bytes_per_launch"] == int(8 * (100e6 + 2e6))
    assert bench.traffic_for("k", path=str(out)) == 8 * (100e6 + 2e6)
    d = json.loads(out.read_text())
    d["k"]["source_sha256"] = "0" * 64
    out.write_text(json.dumps(d))
    assert bench.traffic_for("k", path=str(out)) is None
    assert bench.traffic_for("missing", path=str(out)) is None


def test_launch_count_of_default_step():
    bench = _bench()

    class G:
        dims, periods = (2, 2, 2), (1, 0, 0)
    assert bench.grid_launches_per_step(G(), "f64", True) == 3
    assert bench.grid_launches_per_step(G(), "f32", True) == 2
    G.dims, G.periods = (1, 1, 1), (0, 0, 0)
    assert bench.grid_launches_per_step(G(), "f64", True) == 2
