"""The N > 1 path of bench.py on the CPU with the gloo backend (world size 2):
ranks work on disjoint streams, the job time is the slowest rank's, the
throughput counts every rank's frames, and the reference arm runs on rank 0
only."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [10.0, 25.0][rank]
    job_ms = bench.max_over_ranks(local_ms, world, "cpu")
    value = bench.job_throughput(world, 4, 1000, job_ms)
    seed = bench.video_for_rank(rank).spec.seed
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"job_ms": job_ms, "value": value, "seed": seed}, f)


def test_two_ranks_gloo(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    assert r[0]["job_ms"] == r[1]["job_ms"] == 25.0          # the slowest rank sets the job time
    assert r[0]["value"] == pytest.approx(2 * 4 * 1000 / 0.025)
    assert r[0]["seed"] != r[1]["seed"]                       # disjoint streams


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(1, 2, 500, 100.0) == pytest.approx(10000.0)


def test_reference_arm_only_on_rank_zero(capsys):
    class A:
        start, warmup, steps, gpus = 21, 1, 1, 2
    assert bench.run_reference(A(), 1, 2) is None
    assert capsys.readouterr().out == ""
