"""The multi-GPU form of the benchmark is independent replicas: each rank draws
its own Philox seeds, and the job's rate is every rank's draws over the slowest
rank's time. The host side of that (seed ranges, max-over-ranks time, rate) on
two gloo ranks on the CPU, with one rank slower than the other."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    from oracle import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    steps = 40
    ms_local = [12.5, 30.0][rank]
    ms = bench.job_time_ms(ms_local, world)
    rate = bench.job_rate(steps, world, ms)
    base = bench.replica_seed_base(rank)
    seeds = list(range(base, base + steps))
    u0 = O.uniforms(seeds[0], 0, 8).tolist()
    q.put((rank, ms, rate, seeds, u0))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_rate_and_disjoint_seeds():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, ms, rate, seeds, u0 in out:
        assert ms == 30.0                      # the slowest rank's time
        assert abs(rate - 2 * 40 / 0.030) < 1e-9
    assert not set(out[0][3]) & set(out[1][3])  # disjoint seed ranges
    assert out[0][4] != out[1][4]               # hence different uniforms
