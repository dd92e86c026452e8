"""Host logic of bench.py's replicated N > 1 run, on CPU with the gloo backend.

Every (junction, energy, channel) solve is independent, so N GPUs run N replicas with
no data-path collective; the one exchange is the whole-job figure: the slowest rank's
elapsed time and the units all ranks processed.  Two gloo ranks stand in for two GPUs.
"""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # uneven ranks: elapsed 10, 15, ... ms and 100, 101, ... units
        got = bench.reduce_over_ranks(dist, torch.device("cpu"), 10.0 + 5.0 * rank, 100 + rank)
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = dict(out.get(timeout=10) for _ in range(world))
    # every rank sees the slowest rank's time and the summed units
    for r in range(world):
        assert res[r] == (15.0, 201.0), res


def test_reduce_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(None, None, 12.5, 7) == (12.5, 7.0)


def test_reference_arm_other_ranks_exit_without_work():
    # under torchrun only rank 0 times the oracle and prints; the others exit 0 at once
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


if __name__ == "__main__":
    pytest.main([__file__, "-q"])
