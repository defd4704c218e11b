"""Sharding one batch over ranks (host logic, CPU): contiguous ranges of
whole systems balanced by DOF count, sub-descriptors, and the gather of the
per-rank states into the layout of the whole batch over two gloo ranks."""
import os
import socket

import numpy as np
import torch.distributed as tdist
import torch.multiprocessing as mp

import workloads
from oracle import OracleSystems
from paper_2311_18126_gb300 import shard


def _dofs(desc, part):
    npr = np.asarray(desc["nodes_per_rod"])
    return int(np.sum(4 * npr[part[0]:part[1]] - 1))


def test_partition_covers_every_rod_once_and_balances_dofs():
    desc, _, _ = workloads.uneven_rods(n_rods=4096, seed=2)
    npr = np.asarray(desc["nodes_per_rod"])
    total = int(np.sum(4 * npr - 1))
    for n in (1, 2, 3, 8, 64):
        parts = shard.partition(desc, n)
        assert len(parts) == n and parts[0][0] == 0 and parts[-1][1] == len(npr)
        assert all(parts[k][1] == parts[k + 1][0] for k in range(n - 1))
        # each rank within one rod's DOFs of its share (rods are the systems)
        worst = max(abs(_dofs(desc, p) - total / n) for p in parts)
        assert worst <= np.max(4 * npr - 1), (n, worst)


def test_partition_never_cuts_a_system():
    desc, _, _ = workloads.star_robots(n_robots=37, seed=3)
    sysid = shard.rod_systems(desc)
    assert sysid.max() + 1 == 37
    for n in (2, 5, 36, 40):
        parts = shard.partition(desc, n)
        for (b, e) in parts:
            if b < e:
                assert b == 0 or sysid[b] != sysid[b - 1]
                assert e == len(sysid) or sysid[e] != sysid[e - 1]
        # more ranks than systems: the surplus ranks get empty ranges
        assert sum(1 for (b, e) in parts if e > b) == min(n, 37)
    # one contact group is one system: two ranks, one gets everything
    desc, _, _ = workloads.gripper(n_rods=3, N=10)
    parts = shard.partition(desc, 2)
    assert sorted(e - b for (b, e) in parts) == [0, 3]


def test_sub_descriptors_reproduce_the_batch_state_layout():
    # star robots: joints renumbered per shard; the oracle built on each
    # shard starts from the slice of the whole batch's state
    desc, params, _ = workloads.star_robots(n_robots=5, seed=3, nodes_per_limb=6)
    full = OracleSystems(desc, params).get_state()[0]
    parts = shard.partition(desc, 3)
    pieces = [OracleSystems(shard.sub_descriptor(desc, b, e), params).get_state()[0]
              for (b, e) in parts]
    np.testing.assert_array_equal(np.concatenate(pieces), full)
    np.testing.assert_array_equal(shard.initial_state(desc), full)
    for (off, n), piece in zip(shard.layout_ranges(desc, parts), pieces):
        np.testing.assert_array_equal(full[off:off + n], piece)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        desc, params, kbar = workloads.uneven_rods(n_rods=6, seed=2, n_min=8, n_max=14)
        parts = shard.partition(desc, ws)
        b, e = parts[rank]
        k0, k1 = shard.kbar_ranges(desc, parts)[rank]
        o = OracleSystems(shard.sub_descriptor(desc, b, e), params)
        o.set_natural_curvature(0, e - b, kbar[k0:k1])
        o.step(2)
        q = shard.gather_states(o.get_state()[0], desc, parts)
        if rank == 0:
            out["q"] = q
            out["parts"] = parts
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_step_their_shards_and_gather_the_batch():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True)
        q, parts = out["q"], out["parts"]
    assert all(e > b for (b, e) in parts)
    # the same two steps of the whole batch on one rank
    desc, params, kbar = workloads.uneven_rods(n_rods=6, seed=2, n_min=8, n_max=14)
    o = OracleSystems(desc, params)
    o.set_natural_curvature(0, 6, kbar)
    o.step(2)
    np.testing.assert_array_equal(q, o.get_state()[0])
