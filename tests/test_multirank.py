"""The multi-GPU bench path on CPU: two gloo ranks, each with its own seeded
batch (weak scaling), the slowest rank's time over all ranks, and the
whole-job rate; no collective on the data path."""
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
        desc, _, _ = workloads.uneven_rods(n_rods=8, seed=bench.rank_seed(r))
        t_local = 1.0 + r  # rank 1 is the slow one
        tmax = bench.max_over_ranks(t_local, w)
        out[r] = (int(np.sum(desc["nodes_per_rod"])), tmax, bench.job_rate(w, 8, 10, tmax))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    # independent batches per rank
    assert res[0][0] != res[1][0]
    # both ranks see the slowest rank's time, and the rate counts all ranks
    assert res[0][1] == res[1][1] == 2.0
    assert res[0][2] == res[1][2] == 2 * 8 * 10 / 2.0
