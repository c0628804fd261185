"""The multi-GPU path of bench.py is N independent replicas (the step has no
exchange between grids; no collective on the data path).  Its host logic runs
here on CPU ranks over gloo: the job's throughput is every rank's cells over the
slowest rank's time, the same on every rank; the reference arm does its work on
rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    local_ms = [40.0, 55.0, 47.0][rank]
    value, ms = bench.replica_throughput(torch, local_ms, cells=1 << 20, steps=100, world=world, device="cpu")
    q.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_throughput_max_over_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    slowest = max([40.0, 55.0, 47.0][:world])
    want = world * (1 << 20) * 100 / (slowest * 1e-3) / 1e6
    for _, value, ms in got:
        assert ms == slowest
        assert value == pytest.approx(want, rel=1e-12)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.replica_throughput(torch, 10.0, cells=1000, steps=10, world=1, device="cpu")
    assert ms == 10.0 and value == pytest.approx(1000 * 10 / 0.01 / 1e6)


def test_reference_arm_prints_the_workload_config():
    """Both arms print the same workload config (the driver compares them); the
    oracle's sample and the GPU launch shape sit in their own keys."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    args = bench.parse_args(["--steps", "1", "--warmup", "1"])
    assert line["config"] == bench.workload_config(args, bench.WORKLOADS[args.workload], 1)
    assert line["impl"] == "reference" and line["launch"]["precision"] == "fp64"
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
