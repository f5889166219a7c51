"""The bench's multi-rank logic on CPU ranks (gloo, world size 2): the timing
is the maximum over ranks, every rank agrees on it, the job's throughput
counts every rank's replica, and the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        bench.barrier(ws)
        ms = bench.barrier_max(local_ms, ws)
        rate = bench.job_rate(1000.0, ms, ws)
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as fh:
            json.dump({"ms": ms, "rate": rate}, fh)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    got = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(ws)]
    for g in got:
        assert g["ms"] == 15.0
        assert g["rate"] == pytest.approx(1000.0 * ws / 15e-3)


def test_job_rate_of_one_rank_is_its_own_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.barrier_max(3.5, 1) == 3.5
    assert bench.job_rate(500.0, 250.0, 1) == pytest.approx(2000.0)


def test_reference_arm_prints_on_rank_zero_only():
    outs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
        r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                            "--n-side", "8", "--steps", "1", "--warmup", "0",
                            "--ref-sample", "2"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr
        outs.append(r.stdout.strip())
    assert outs[1] == ""
    line = json.loads(outs[0].splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
