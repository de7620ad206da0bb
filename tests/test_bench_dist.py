"""The multi-rank logic of bench.py on CPU: two gloo ranks, max-over-ranks
timing and the whole-job aggregate (weak scaling, replicas only)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    mx = bench.max_over_ranks(ms)
    value = bench.whole_job_value(1000, 4, mx, world)
    out[rank] = (mx, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        mx, value = out[r]
        assert mx == 15.0
        assert value == pytest.approx(2 * 1000 * 4 / 0.015)


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_value(10, 2, 1.0, 1) == pytest.approx(20000.0)


def test_traffic_guard_tracks_sources():
    import bench
    t = bench.render_traffic()
    assert t is None or t == bench.RENDER_TRAFFIC["bytes"]


def test_reference_arm_under_two_ranks_prints_one_line():
    """`--impl reference` launched as two ranks: rank 0 alone times the
    oracle and prints the line, the other rank exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 1
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
