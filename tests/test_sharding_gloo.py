"""The multi-rank path on CPU: two gloo ranks each simulate their contiguous share of trajectory ids
(with the FP64 oracle standing in for each rank's GPU) and combine them with the sharding helpers' all-
reduces; the ensemble mean and the summed gradient equal those of one process over all ids, because
every random number is keyed by the global trajectory id. Also checks the partition and the max/sum
reductions the benchmark uses. Cases: the LINEAR readout of 2A <-> B, the bin readout of the ion
channel with the exact and with the soft forward, and the GRN classifier (hard and soft) sharded by images."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2602_19775_gb300.shard import (global_ensemble_mean, global_gradient, max_over_ranks, shard_range,
                                          total_over_ranks)


def test_shard_range_partitions_contiguously():
    for n in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            spans = [shard_range(n, r, world) for r in range(world)]
            assert sum(c for _, c in spans) == n
            pos = 0
            for off, c in spans:
                assert off == pos
                pos += c
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case(kind, n_total):
    """(network spec, log rates, x0, t_end, sample times, observed species, readout, selector) of a case."""
    import ssa_workloads as W
    from oracle import native
    if kind == "c2_linear":
        wl = W.config_c2(n_traj=n_total)
        return wl.net, wl.log_rates, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, native.LINEAR, "gumbel"
    net = W.ion_channel_coi()
    ts = W.uniform_sample_grid(8.0, 40)
    sel = "soft" if kind == "ion_bin_soft" else "gumbel"
    return net, net.log_rates, net.x0, 8.0, ts, np.array([1], np.int32), native.BIN, sel


def _rank_main(rank, world, port, n_total, kind, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import native
        net, theta, x0, t_end, ts, obs_sp, readout, sel = _case(kind, n_total)
        off, cnt = shard_range(n_total, rank, world)
        dl = np.full((cnt, len(ts), len(obs_sp)), 1.0 / n_total)
        r = native.run(net, theta, x0, cnt, t_end, ts, obs_sp, 5, readout, max_steps=4096, traj_offset=off, dl_dobs=dl,
                       temperature=0.5, n_threads=1, selector=sel)
        mean = global_ensemble_mean(torch.tensor(r.obs))
        grad = global_gradient(torch.tensor(r.dtheta.sum(0)))
        t = max_over_ranks(1.0 + rank)
        steps = total_over_ranks(int(r.draws.sum()))
        if rank == 0:
            out.put((mean.numpy(), grad.numpy(), t, steps))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["c2_linear", "ion_bin", "ion_bin_soft"])
def test_two_gloo_ranks_reproduce_one_process(kind):
    from oracle import native
    n_total = 301  # uneven split
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, n_total, kind, q)) for r in range(2)]
    for p in procs:
        p.start()
    mean, grad, t, steps = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    net, theta, x0, t_end, ts, obs_sp, readout, sel = _case(kind, n_total)
    dl = np.full((n_total, len(ts), len(obs_sp)), 1.0 / n_total)
    r = native.run(net, theta, x0, n_total, t_end, ts, obs_sp, 5, readout, max_steps=4096, dl_dobs=dl, temperature=0.5,
                   n_threads=1, selector=sel)
    np.testing.assert_allclose(mean, r.obs.mean(0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(grad, r.dtheta.sum(0), rtol=1e-12, atol=1e-15)
    assert t == 2.0
    assert steps == int(r.draws.sum())


def _grn_case():
    """A small GRN classifier (5 inputs, 4 hidden genes, 3 outputs) on 7 synthetic images x 16 trajectories."""
    from ssa_workloads import grn as G
    p = G.grn_params(seed=1, n_in=5, n_hid=4, n_out=3, w1_scale=0.02, w2_scale=0.5)
    p.b1[:] = [0.3, -0.5, 1.0, 0.0]
    p.b2[:] = [0.2, -0.1, 0.4]
    x = np.random.default_rng(3).integers(0, 256, size=(7, 5)).astype(np.int32)
    return p, x, 16, 4.0, np.array([2.0, 4.0])


def _flat_grads(res, x, tpi):
    g = res.grads(x, tpi)
    return np.concatenate([np.ravel(g[k]) for k in ("W1", "b1", "W2", "b2", "log_d")])


def _grn_rank_main(rank, world, port, soft, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import native
        p, x, tpi, t_end, ts = _grn_case()
        img_off, img_cnt = shard_range(x.shape[0], rank, world)  # whole images per rank
        xs = x[img_off:img_off + img_cnt]
        n_all = x.shape[0] * tpi
        dl = np.full((img_cnt * tpi, len(ts), p.n_out), 1.0 / n_all)
        r = native.grn_run(p, xs, tpi, t_end, ts, 9, max_steps=4096, traj_offset=img_off * tpi, dl_dobs=dl,
                           temperature=0.7, n_threads=1, soft=soft)
        mean = global_ensemble_mean(torch.tensor(r.obs))
        grad = global_gradient(torch.tensor(_flat_grads(r, xs, tpi)))
        if rank == 0:
            out.put((mean.numpy(), grad.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("soft", [False, True], ids=["grn_hard", "grn_soft"])
def test_two_gloo_ranks_shard_the_grn_by_images(soft):
    """The GRN classifier sharded by whole images (trajectory ids img_off * traj_per_img onwards on each
    rank): the ensemble mean of the outputs and every parameter gradient equal one process's."""
    from oracle import native
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grn_rank_main, args=(r, 2, port, soft, q)) for r in range(2)]
    for p in procs:
        p.start()
    mean, grad = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    p, x, tpi, t_end, ts = _grn_case()
    n_all = x.shape[0] * tpi
    dl = np.full((n_all, len(ts), p.n_out), 1.0 / n_all)
    r = native.grn_run(p, x, tpi, t_end, ts, 9, max_steps=4096, dl_dobs=dl, temperature=0.7, n_threads=1, soft=soft)
    np.testing.assert_allclose(mean, r.obs.mean(0), rtol=1e-12, atol=1e-12)
    ref = _flat_grads(r, x, tpi)
    np.testing.assert_allclose(grad, ref, rtol=1e-10, atol=1e-14 * np.abs(ref).max())
    assert np.abs(ref).max() > 0
