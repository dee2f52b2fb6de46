"""The multi-GPU path on the CPU, through the product's own exchange functions
(paper_1504_02776_gb300.shards): two gloo ranks trace their own neutron-id shards with the
oracle standing in for the kernels.

  - Forward: shards.reduce_sum sums the ranks' histograms and tallies; the result equals one
    run over the union of the shards (a neutron's history depends only on (seed, sim_id, id)).
  - Gradient: shards.sharded_gradient runs each rank's forward, sums the histograms, runs each
    rank's adjoint on the summed histogram and sums the gradients; loss and gradient equal
    those of one run over all the ids, on every rank.
Also checks that the shard helpers cover the ids once."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import mcv_inputs as mi
from paper_1504_02776_gb300.shards import reduce_sum, shard, sharded_gradient, split

N_PER_RANK = 1500


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _grad_case():
    import oracle
    det = mi.tube_detector(n_tof=40, packs=(38, 39, 38), pixels_per_tube=16)
    wl = mi.config2(n=3001).replace(detector=det)
    tw = wl.replace(sqe=mi.SqeGrid(mi.sqe_table(omega_scale=1.05)), seed=1)
    ref = oracle.trace(tw, packets=False)["hist"]
    c = 1e4 / ref.sum()
    return wl, mi.poisson_target(ref, c, seed=2), c


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    # forward: each rank's shard, then the sum over the ranks
    wl = mi.config1(n=N_PER_RANK)
    first, n = shard(rank, world, N_PER_RANK)
    r = oracle.trace(wl, first_id=first, n=n, packets=False)
    h = torch.from_numpy(r["hist"].copy())
    t = torch.from_numpy(r["tallies"].copy())
    reduce_sum([h, t])
    # gradient of a run split over the ranks (the oracle standing in for the kernels)
    gw, target, c = _grad_case()

    def forward(f, m, hist):
        hist += torch.from_numpy(oracle.trace(gw, first_id=f, n=m, packets=False)["hist"])

    def adjoint(f, m, hist):
        out = oracle.adjoint(gw, hist.numpy(), target, c, first_id=f, n=m)
        return {"loss": out["loss"], "dsqe": torch.from_numpy(out["dsqe"].ravel().copy()),
                "dsig": torch.from_numpy(out["dsig"].copy())}

    g = sharded_gradient(forward, adjoint, torch.zeros(gw.detector.n_bins, dtype=torch.float64),
                         rank, world, gw.n)
    np.save(os.path.join(out_dir, "dsqe_%d.npy" % rank), g["dsqe"].numpy())
    np.save(os.path.join(out_dir, "dsig_%d.npy" % rank), g["dsig"].numpy())
    np.save(os.path.join(out_dir, "loss_%d.npy" % rank), np.array([g["loss"]]))
    if rank == 0:
        np.save(os.path.join(out_dir, "hist.npy"), h.numpy())
        np.save(os.path.join(out_dir, "tallies.npy"), t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_add_up_to_one_run(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import oracle
    h = np.load(tmp_path / "hist.npy")
    t = np.load(tmp_path / "tallies.npy")
    ref = oracle.trace(mi.config1(n=world * N_PER_RANK), first_id=0, packets=False)
    assert ref["tallies"][oracle.T_NDET] > 0
    assert np.allclose(h, ref["hist"], rtol=1e-12, atol=0.0)
    assert np.allclose(t, ref["tallies"], rtol=1e-12, atol=0.0)
    # the split gradient equals that of one run over every id, on both ranks
    gw, target, c = _grad_case()
    g = oracle.grad(gw, target, c)
    ref_s = g["dsqe"].ravel()
    assert np.abs(ref_s).max() > 0
    for r in range(world):
        loss = float(np.load(tmp_path / ("loss_%d.npy" % r))[0])
        assert abs(loss - g["loss"]) <= 1e-12 * g["loss"]
        np.testing.assert_allclose(np.load(tmp_path / ("dsig_%d.npy" % r)), g["dsig"], rtol=1e-11)
        dsqe = np.load(tmp_path / ("dsqe_%d.npy" % r))
        assert np.abs(dsqe - ref_s).max() <= 1e-11 * np.abs(ref_s).max()


def test_reduce_sum_is_a_no_op_in_one_process():
    a = torch.ones(3)
    assert reduce_sum([a])[0] is a and torch.equal(a, torch.ones(3))


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
