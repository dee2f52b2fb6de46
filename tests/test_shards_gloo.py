"""The multi-GPU path on the CPU: two gloo ranks trace their own neutron-id shards with the
oracle and sum their histograms and tallies with an all-reduce; the result equals one run
over the union of the shards (the property the sharded GPU run relies on: a neutron's history
depends only on (seed, sim_id, id)).  Also checks that the shard helpers cover the ids once."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import mcv_inputs as mi
from paper_1504_02776_gb300.shards import shard, split

N_PER_RANK = 1500


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    wl = mi.config1(n=N_PER_RANK)
    first, n = shard(rank, world, N_PER_RANK)
    r = oracle.trace(wl, first_id=first, n=n, packets=False)
    h = torch.from_numpy(r["hist"].copy())
    t = torch.from_numpy(r["tallies"].copy())
    dist.all_reduce(h, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(os.path.join(out_dir, "hist.npy"), h.numpy())
        np.save(os.path.join(out_dir, "tallies.npy"), t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_add_up_to_one_run(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    h = np.load(tmp_path / "hist.npy")
    t = np.load(tmp_path / "tallies.npy")
    import oracle
    ref = oracle.trace(mi.config1(n=world * N_PER_RANK), first_id=0, packets=False)
    assert ref["tallies"][oracle.T_NDET] > 0
    assert np.allclose(h, ref["hist"], rtol=1e-12, atol=0.0)
    assert np.allclose(t, ref["tallies"], rtol=1e-12, atol=0.0)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shards_cover_the_ids_once(world):
    n = 1000
    got = []
    for r in range(world):
        f, m = shard(r, world, n, first_id=7)
        got.extend(range(f, f + m))
    assert got == list(range(7, 7 + world * n))
    total = 1003
    got = []
    for r in range(world):
        f, m = split(r, world, total, first_id=5)
        got.extend(range(f, f + m))
    assert got == list(range(5, 5 + total))
    with pytest.raises(ValueError):
        shard(world, world, n)
