"""The multi-process (replica) path on CPU: two gloo ranks, as torchrun would start them."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1309_6250_gb300 import inputs, replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    r, ws, local = replicas.env_rank_world()
    dist.init_process_group("gloo", rank=r, world_size=ws)
    cell = inputs.CELLS["c2"]
    pos = replicas.rank_positions(cell.lattice, 64, cell.pos_seed, r)
    # each rank's slowest time is its own; the job time is the maximum
    elapsed = 1.0 + r
    job_s = replicas.max_over_ranks(elapsed, dist)
    gathered = [torch.zeros(64 * 3, dtype=torch.float64) for _ in range(ws)]
    dist.all_gather(gathered, torch.from_numpy(pos.reshape(-1)))
    dist.barrier()
    out[r] = (r, ws, local, job_s, replicas.job_throughput(1000.0, ws, job_s),
              [g.numpy().copy() for g in gathered])
    dist.destroy_process_group()


def test_two_gloo_ranks_replica_logic():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    res = dict(out)
    assert sorted(res) == [0, 1]
    for r in range(world):
        rr, ws, local, job_s, thr, gathered = res[r]
        assert (rr, ws, local) == (r, world, r)
        assert job_s == 2.0                       # max over ranks
        assert thr == pytest.approx(1000.0 * 2 / 2.0)
        # rank 0 keeps the workload's positions; rank 1 has its own, different walkers
        cell = inputs.CELLS["c2"]
        np.testing.assert_array_equal(gathered[0], inputs.positions(cell.lattice, 64, cell.pos_seed).reshape(-1))
        assert not np.allclose(gathered[0], gathered[1])


def test_single_process_defaults():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.position_seed(2000, 0) == 2000
    assert replicas.job_throughput(10.0, 4, 2.0) == 20.0
