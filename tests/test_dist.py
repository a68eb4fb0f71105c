"""The multi-GPU bench path's host logic with two gloo ranks on the CPU: rendezvous on
127.0.0.1, the max of per-rank times that every rank reports, the barriers, and distinct
sources per rank (sources are sharded across ranks; no data crosses them)."""
import multiprocessing as mp
import os
import socket

import numpy as np


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), CUDA_VISIBLE_DEVICES="")
    try:
        import torch.distributed as dist
        import bench
        import tt_inputs as I
        r, w = bench.dist_init()
        assert (r, w) == (rank, world)
        bench.dist_barrier(w)
        m = bench.dist_max(10.0 * (rank + 1), w)
        src = I.random_sources(I.GridSpec(9, 9, 9, 0.0, 10.0, 0.0, 1.0, 0.0, 1.0), 4, (1.0, 9.0),
                               np.random.default_rng(bench.rank_seed(rank)))
        bench.dist_barrier(w)
        dist.destroy_process_group()
        q.put((rank, m, src.tolist(), None))
    except Exception as e:  # reported to the parent
        q.put((rank, None, None, repr(e)))


def test_two_gloo_ranks_share_max_time_and_shard_sources():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, m, src, err = q.get(timeout=120)
        assert err is None, err
        out[rank] = (m, np.array(src))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 20.0          # every rank reports the slowest rank's time
    assert not np.array_equal(out[0][1], out[1][1])  # different sources on each rank
