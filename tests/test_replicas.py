"""bench.py's multi-GPU mode is replicas only (the path shards by scene or partition
with no data-path collective here): its host logic is exercised with two gloo ranks on
the CPU -- the max-over-ranks timing, the whole-job throughput, and the reference arm
running on rank 0 alone."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, w, "cpu")
    dist.barrier()
    out.put((r, w, lr, ms, bench.job_throughput(w, 1000, 10, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    for r in res:
        assert r[3] == 15.0                       # the slower rank's 15 ms, on both ranks
        assert r[4] == pytest.approx(2 * 1000 * 10 / 15e-3)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.run_reference(bench.parse([]), rank=1, world=2) == 0


def test_reference_arm_prints_its_line(capsys):
    """The reference arm (the oracle on the host cores, a bounded sample of the workload)
    prints one JSON line with the contract's keys."""
    import json

    sys.path.insert(0, ROOT)
    import bench

    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0", "--n-pts", "20000",
                        "--reference-seconds", "6"])
    assert bench.run_reference(args, rank=0, world=1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
