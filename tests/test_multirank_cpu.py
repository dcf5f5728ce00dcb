"""The N > 1 host path of bench.py on CPU: two gloo ranks (replicas, no data
collective) agree on the slowest rank's time and report the whole-job
rate; the reference arm runs on rank 0 only while the other rank waits at
the barrier and exits."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    t = bench.max_over_ranks(0.5 + rank, dist, "cpu")      # rank 1 is the slow one
    out[rank] = (t, bench.whole_job_rate(ws, 1000.0, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_the_whole_job_rate():
    ws = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == res[1] == (1.5, pytest.approx(2 * 1000.0 / 1.5))


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(0.25, None, "cpu") == 0.25
    assert bench.whole_job_rate(1, 10.0, 2.0) == 5.0


def test_reference_arm_under_two_ranks_prints_one_line_from_rank_zero():
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "3"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
