"""The N > 1 bench path on CPU: two gloo ranks (no GPU).

Frames shard across ranks with no data-path collective (each rank owns its
trajectory, weak scaling); the only exchange is the max over ranks of the
step time, and `value` counts the atom-frames of all ranks.
"""

import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    t = bench.max_over_ranks(dist, 10.0 + rank, torch.device("cpu"), world)
    frames, _, _ = synth.water_bulk(n_frames=2, n_side=4, L=12.42, seed_k=bench.shard_seed_k(rank))
    q.put((rank, t, float(frames[1].sum()), bench.job_units(2, 192, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, u0), (r1, t1, s1, u1) = res
    assert t0 == t1 == 11.0             # max over ranks
    assert s0 != s1                     # each rank evaluates its own trajectory
    assert u0 == u1 == 2 * 192 * world  # whole-job atom-frames
