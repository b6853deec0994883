"""The benchmark's multi-process path on CPU (gloo, world size 2): replicas
only, so the ranks share nothing but the barrier and the max-over-ranks
timing; rank 0 alone prints the result line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, local = bench.dist_init("gloo")
    assert (w, r, local) == (world, rank, rank)
    dist.barrier()
    t = bench.max_over_ranks(1.0 + 0.5 * rank, w, "cpu")      # rank k took 1 + k/2 s
    rate = bench.job_rate(1000, w, t)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"t": t, "rate": rate}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r in res:
        assert r["t"] == 1.5                    # the slowest rank's time on every rank
        assert r["rate"] == 1000 * 2 / 1.5      # units of all ranks / that time


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert bench.job_rate(10, 1, 2.0) == 5.0


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` launched like the multi-GPU runs: rank 0
    times the oracle and prints one line, rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3", "--workload", "eremd_8x2048"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, env=env, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    # the reference line reports the same config dict as the GPU arm would
    sys.path.insert(0, ROOT)
    import bench
    b = bench.workload("eremd_8x2048")
    assert line["config"] == json.loads(json.dumps(bench.bench_config("eremd_8x2048", b, b.pairs_per_eval())))
    assert "2 BAOAB MD steps" in line["sample"]
