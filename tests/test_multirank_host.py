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


def _rank_chain(rank, world, port, out_dir):
    # each rank runs the method (the CPU oracle's chain) on its own stream of
    # the tiny workload against the replicated index; the only collectives
    # are the job time and a checksum of every rank's fields
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    import synth
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.WORKLOADS["tiny"]
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    oix = oracle.Index(R, KP)
    video = bench.video_for_rank(rank, w.video)
    import time
    t0 = time.perf_counter()
    prev, fields = None, []
    for t in range(3):
        a, _, _, _ = oracle.riann_frame(oix, video.frame(t), prev, ring_limit=w.n // 8)
        fields.append(a)
        prev = a
    ms = 1000.0 * (time.perf_counter() - t0)
    local = int(sum(int(f.astype(np.int64).sum()) for f in fields))
    tot = torch.tensor([local], dtype=torch.int64)
    dist.all_reduce(tot)
    job_ms = bench.max_over_ranks(ms, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"f{rank}.npy"), np.stack(fields))
    with open(os.path.join(out_dir, f"c{rank}.json"), "w") as f:
        json.dump({"local": local, "total": int(tot.item()), "ms": ms, "job_ms": job_ms,
                   "seed": video.spec.seed}, f)


def test_two_ranks_run_their_own_streams(tmp_path):
    import numpy as np
    port = _free_port()
    mp.spawn(_rank_chain, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"c{k}.json")) for k in range(2)]
    f = [np.load(tmp_path / f"f{k}.npy") for k in range(2)]
    assert r[0]["seed"] != r[1]["seed"]
    assert not np.array_equal(f[0], f[1])                    # disjoint streams, different fields
    assert r[0]["total"] == r[1]["total"] == r[0]["local"] + r[1]["local"]
    assert r[0]["job_ms"] == r[1]["job_ms"] == max(r[0]["ms"], r[1]["ms"])
    # rank 1's stream run alone gives its fields: no state crosses ranks
    import oracle
    import synth
    w = synth.WORKLOADS["tiny"]
    R = synth.workload_reference(w)
    oix = oracle.Index(R, synth.workload_keypoints(w, R))
    video = bench.video_for_rank(1, w.video)
    prev = None
    for t in range(3):
        a, _, _, _ = oracle.riann_frame(oix, video.frame(t), prev, ring_limit=w.n // 8)
        assert np.array_equal(a, f[1][t])
        prev = a


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
