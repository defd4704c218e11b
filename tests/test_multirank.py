"""The multi-GPU bench path on CPU: two gloo ranks, each with its shard of
one seeded batch twice the one-GPU size (weak scaling), the slowest rank's
time over all ranks, and the whole-job rate; no collective on the data
path."""
import os
import socket

import numpy as np
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

import bench
import workloads


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, _ = bench.dist()
        desc, _, kbar, total = bench.shard_of_batch(
            lambda n: workloads.uneven_rods(n_rods=8 * n, seed=2), w, r)
        t_local = 1.0 + r  # rank 1 is the slow one
        tmax = bench.max_over_ranks(t_local, w)
        out[r] = (tuple(desc["nodes_per_rod"]), len(kbar), total, tmax,
                  bench.job_rate(total, 10, tmax))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    # the two shards are the two halves of one 16-rod batch
    whole, _, _ = workloads.uneven_rods(n_rods=16, seed=2)
    assert res[0][0] + res[1][0] == tuple(whole["nodes_per_rod"])
    assert res[0][1] + res[1][1] == int(np.sum(np.asarray(whole["nodes_per_rod"]) - 2))
    assert res[0][2] == res[1][2] == 16
    # both ranks see the slowest rank's time, and the rate counts all ranks
    assert res[0][3] == res[1][3] == 2.0
    assert res[0][4] == res[1][4] == 16 * 10 / 2.0
