"""The N>1 benchmark path runs independent replicas: each rank simulates
its own shot, and gloo is used only for the timing barrier and the
max-over-ranks time.  Run as two CPU processes (world size 2, gloo)."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2205_07976_gb300 import workloads as W
    w, r, local, pg = bench.dist_setup(None)
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(pg)
    my_time = 1.0 + 0.25 * rank
    t = bench.max_over_ranks(pg, my_time)
    shot = W.single_shot_small(seed=1 + rank)
    out.put((rank, t, shot.axes.tobytes(), shot.pixel_steps))
    pg.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_distinct_shots():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # every rank sees the slowest rank's time
    assert [t for _, t, _, _ in res] == [1.25, 1.25]
    # replicas simulate different shots of the same size
    assert res[0][2] != res[1][2]
    assert res[0][3] == res[1][3]
    # whole-job rate = units of all ranks / slowest time
    units = sum(ps_ for _, _, _, ps_ in res)
    assert np.isclose(units / res[0][1], 2 * res[0][3] / 1.25)
