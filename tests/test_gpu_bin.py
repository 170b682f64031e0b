"""GPU tests of the exact bin-averaged readout (arXiv 2602.19775, Section 4.4) against the FP64 oracle:
bin averages element by element on the same seeded trajectories, the straight-through gradient through
them, the ensemble means of the ion-channel workload (262,144 trajectories, 800 bins of 0.01 ms) against
the master equation averaged over each bin, and the input rules and limits of the readout.

Tolerance of a bin average on a trajectory whose event sequence matches the oracle's: every event time
inside the bin may be off by the FP32 clock tolerance, moving a jump of at most max|v| by that much, and
the binary32 sum over the bin's pieces adds a few roundings of the largest count:
    |obs_gpu - obs_oracle| <= (n_events * max|v| * tol(t_s) + (n_events + 4) * 4 eps32 * max X * D_s) / D_s.
"""
import numpy as np
import pytest
import torch

import ssa_workloads as W
from oracle import cme, native

from test_gpu_parity import EPS32, GRAD_RTOL, _bracket_agreement, _clock_tol, _compare_events, _theta32

pytestmark = pytest.mark.gpu
BIN = native.BIN


@pytest.fixture(scope="module")
def S():
    from paper_2602_19775_gb300 import ssa
    ssa._lib.lib()
    return ssa


def _lo(ts):
    return np.concatenate([[0.0], np.asarray(ts)[:-1]])


def _run_both(S, net, n, t_end, ts, obs_sp, seed, dl=None, T=1.0, max_steps=4096, specialize=True, K=64, tpt=0):
    t32, t64 = _theta32(net.log_rates)
    snet = S.Network(net)
    fw = S.forward(snet, torch.tensor(t32, device="cuda"), n, net.x0, t_end, ts, obs_sp, seed, readout="bin",
                   record=True, max_steps=max_steps, specialize=specialize, ckpt_interval=K, threads_per_traj=tpt)
    torch.cuda.synchronize()
    orc = native.run(net, t64, net.x0, n, t_end, ts, np.asarray(obs_sp, np.int32), seed, BIN, max_steps=max_steps,
                     dl_dobs=dl, temperature=T, ev_cap=max_steps)
    return snet, fw, orc, fw.run.events(max_steps).cpu().numpy()


def _check_obs(net, fw, orc, same, ts, obs_sp):
    V = net.stoich_dense()
    vmax = np.abs(V[:, obs_sp]).max(0)
    lo, D = _lo(ts), np.asarray(ts) - _lo(ts)
    obs_g = fw.obs.double().cpu().numpy()
    tol_t = _clock_tol(net.n_reactions, np.asarray(ts))
    worst = 0.0
    for i in np.nonzero(same)[0]:
        t_ev = orc.times[i, :orc.draws[i]]
        xmax = np.abs(orc.obs[i]).max(0) * 2 + 1
        for s in range(len(ts)):
            n_ev = np.sum((t_ev > lo[s] - tol_t[s]) & (t_ev <= ts[s] + tol_t[s]))
            bound = (n_ev * vmax * tol_t[s] + (n_ev + 4) * 4 * EPS32 * xmax * D[s]) / D[s]
            err = np.abs(obs_g[i, s] - orc.obs[i, s])
            assert np.all(err <= bound), (i, s, obs_g[i, s], orc.obs[i, s], bound)
            worst = max(worst, float((err / bound).max()))
    return worst


CASES = {
    "ion_channel": lambda: (W.ion_channel_coi(), 8.0, W.uniform_sample_grid(8.0, 80), [1], 4096),
    "mixed_orders": lambda: (W.mixed_orders_toy(), 6.0, W.uniform_sample_grid(6.0, 11), [0, 1, 2], 1000),
    "dimer": lambda: (W.dimerization_2a_b(0.02, 0.05, 100), 50.0, W.uniform_sample_grid(50.0, 50), [0, 1], 2048),
    "ragged_bins": lambda: (W.mixed_orders_toy(), 5.0, np.array([1e-3, 0.5, 0.5 + 1e-6, 0.75, 3.0, 4.999, 5.0]),
                            [0, 2], 777),
}


@pytest.mark.parametrize("specialize", [True, False])
@pytest.mark.parametrize("case", sorted(CASES))
def test_bin_forward_matches_oracle(S, case, specialize):
    net, t_end, ts, obs_sp, n = CASES[case]()
    snet, fw, orc, gev = _run_both(S, net, n, t_end, ts, obs_sp, 3, specialize=specialize)
    assert fw.run.variant == (2 if specialize else 1)
    assert np.all(fw.status.cpu().numpy() <= 1)
    same = _compare_events(orc, fw, gev, t_end, net.n_reactions)
    _check_obs(net, fw, orc, same, ts, np.asarray(obs_sp))


@pytest.mark.parametrize("case,T", [("ion_channel", 0.5), ("mixed_orders", 0.5), ("dimer", 0.1), ("dimer", 1.0),
                                    ("ragged_bins", 0.3)])
def test_bin_backward_matches_oracle(S, case, T):
    net, t_end, ts, obs_sp, n = CASES[case]()
    dl = W.seeded_dl_dobs(5, n, len(ts), len(obs_sp), scale=1.0 / n)
    snet, fw, orc, gev = _run_both(S, net, n, t_end, ts, obs_sp, 9, dl=dl, T=T, K=16)
    same = _compare_events(orc, fw, gev, t_end, net.n_reactions)
    # an event within the clock tolerance of an edge moves its time derivative to the other bin
    agree = _bracket_agreement(orc, fw, np.asarray(ts), net.n_reactions)
    assert agree.mean() >= 0.99, agree.mean()
    same &= agree
    dl_g = dl.copy()
    dl_g[~same] = 0.0
    g = S.backward(fw, torch.tensor(dl_g, dtype=torch.float32, device="cuda"), T).cpu().numpy().astype(np.float64)
    ref = orc.dtheta[same].sum(0)
    assert fw.run.status_counts()[1] == 0
    rel = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30)
    assert rel < GRAD_RTOL, (rel, g, ref)
    big = np.abs(ref) > 1e-3 * np.linalg.norm(ref)
    np.testing.assert_allclose(g[big], ref[big], rtol=2 * GRAD_RTOL)


def test_ion_channel_bin_means_match_cme(S):
    """The Section 4.4 workload at its size: 2 channels C <-> O -> I, 262,144 trajectories, 800 bins of
    0.01 ms over 8 ms; ensemble means of the open count against the CME law averaged over each bin."""
    net = W.ion_channel_coi()
    ts = W.uniform_sample_grid(8.0, 800)
    n = 262144
    snet = S.Network(net)
    fw = S.forward(snet, torch.tensor(net.log_rates.astype(np.float32), device="cuda"), n, net.x0, 8.0, ts, [1], 17,
                   readout="bin", max_steps=64)
    assert int((fw.status > 1).sum()) == 0
    O = fw.obs[:, :, 0].double()
    m = O.mean(0).cpu().numpy()
    se = (O.std(0) / np.sqrt(n)).cpu().numpy()
    k32 = net.log_rates.astype(np.float32).astype(np.float64)
    states, index = cme.reachable_states(net, net.x0)
    Q = cme.generator(net, k32, states, index)
    p0 = np.zeros(len(states))
    p0[index[tuple(int(v) for v in net.x0)]] = 1.0
    exact = cme.transient_bin_average(Q, p0, ts) @ np.array([x[1] for x in states], dtype=np.float64)
    z = (m - exact) / np.maximum(se, 1e-12)
    # 800 correlated bins: 4.5 SE each keeps the family-wise false-alarm rate under 1%
    assert np.all(np.abs(z) < 4.5), (np.abs(z).max(), int(np.abs(z).argmax()))


def test_bin_autograd_function_matches_backward(S):
    net = W.ion_channel_coi()
    ts = W.uniform_sample_grid(8.0, 40)
    theta = torch.tensor(net.log_rates.astype(np.float32), device="cuda", requires_grad=True)
    target = torch.linspace(0.0, 0.5, 40, device="cuda")[:, None]
    snet = S.Network(net)
    obs = S.simulate(snet, theta, 8192, net.x0, 8.0, ts, [1], 4, readout="bin", temperature=0.5, max_steps=64)
    loss = ((obs.mean(0) - target) ** 2).mean()
    loss.backward()
    fw = S.forward(snet, theta.detach(), 8192, net.x0, 8.0, ts, [1], 4, readout="bin", record=True, max_steps=64)
    assert torch.equal(fw.obs, obs.detach())
    dl = 2.0 * (fw.obs.mean(0) - target) / target.numel() / 8192
    g = S.backward(fw, dl.expand(8192, -1, -1).contiguous(), 0.5)
    torch.testing.assert_close(theta.grad, g, rtol=1e-5, atol=1e-7)


def test_bin_input_rules_and_limits(S):
    net = W.mixed_orders_toy()
    snet = S.Network(net)
    theta = torch.tensor(net.log_rates.astype(np.float32), device="cuda")
    # a path that cannot move: every bin holds the initial state exactly, and the gradient is zero
    frozen = W.network_from_reactions(["A", "B"], [(["A", "B"], ["B"], "k")], rates={"k": 1.0}, x0={"A": 3})
    fnet = S.Network(frozen)
    fw = S.forward(fnet, torch.tensor(frozen.log_rates.astype(np.float32), device="cuda"), 5, frozen.x0, 2.0,
                   [0.5, 1.0, 2.0], [0, 1], 0, readout="bin", record=True)
    assert torch.equal(fw.obs.cpu(), torch.tensor([[3.0, 0.0]] * 3).expand(5, 3, 2))
    assert int(fw.status[0]) == 1
    g = S.backward(fw, torch.ones(5, 3, 2, device="cuda"), 0.5)
    assert torch.count_nonzero(g) == 0
    # empty first bin (t_0 = 0) or a repeated edge: every trajectory is BAD_INPUT
    for ts in ([0.0, 1.0], [0.5, 0.5, 1.0]):
        fw = S.forward(snet, theta, 8, net.x0, 1.0, ts, [0], 0, readout="bin")
        assert torch.all(fw.status == 6), ts
    # the same edges are fine for the HOLD readout
    fw = S.forward(snet, theta, 8, net.x0, 1.0, [0.0, 1.0], [0], 0, readout="hold")
    assert torch.all(fw.status <= 1)
    # more than SSA_BIN_MAX_OBS observables are refused, on every kernel and in the batch
    with pytest.raises(RuntimeError):
        S.forward(snet, theta, 8, net.x0, 1.0, [1.0], [0, 1, 2, 0, 1], 0, readout="bin")
    with pytest.raises(RuntimeError):
        S.forward(snet, theta, 8, net.x0, 1.0, [1.0], [0, 1, 2, 0, 1], 0, readout="bin", threads_per_traj=32)
    with pytest.raises(RuntimeError):
        S.Batch([dict(net=snet, log_rates=theta, n_traj=8, x0=net.x0, t_end=1.0, sample_times=[1.0],
                      obs_species=[0, 1, 2, 0, 1], seed=0)], readout="bin")
    # a batch item's bin edges follow the same rule: an empty first bin makes its trajectories BAD_INPUT
    b = S.Batch([dict(net=snet, log_rates=theta, n_traj=8, x0=net.x0, t_end=1.0, sample_times=[0.0, 1.0],
                      obs_species=[0], seed=0)], readout="bin")
    b.run()
    assert torch.all(b.outputs(0)[1] == 6)
    # empty batch of trajectories
    fw = S.forward(snet, theta, 0, net.x0, 1.0, [0.5, 1.0], [0], 0, readout="bin", record=True)
    assert fw.obs.shape == (0, 2, 1)


@pytest.mark.parametrize("specialize", [True, False])
def test_bin_shared_upstream_gradient_matches_full(S, specialize):
    """A loss on ensemble means gives every trajectory the same dL/dobs; passed once ([S][n_obs], stride 0)
    the adjoint sums it over runs of whole bins by binary64 prefix sums, passed per trajectory it sums
    bin by bin: the two gradients agree to binary32 rounding."""
    net = W.ion_channel_coi()
    ts = W.uniform_sample_grid(8.0, 800)
    snet = S.Network(net)
    theta = torch.tensor(net.log_rates.astype(np.float32), device="cuda")
    n = 65536
    fw = S.forward(snet, theta, n, net.x0, 8.0, ts, [1], 21, readout="bin", record=True, max_steps=64,
                   specialize=specialize)
    g = torch.tensor(W.seeded_dl_dobs(3, 1, 800, 1)[0] / n, dtype=torch.float32, device="cuda")
    shared = S.backward(fw, g, 0.5).double().cpu().numpy()
    full = S.backward(fw, g.expand(n, -1, -1).contiguous(), 0.5).double().cpu().numpy()
    assert np.abs(shared - full).max() <= 1e-4 * np.abs(full).max(), (shared, full)


def test_bin_on_the_generic_runtime_loop_kernels(S):
    """A network above the specialisation limits (M = 30) runs the generic thread kernels with runtime loops
    over the reactions; the bin readout and its gradient still match the oracle."""
    spec = W.random_network(np.random.default_rng(5), n_species_range=(6, 12), n_reactions_range=(30, 30))
    from test_gpu_warp import _pilot_t_end
    t_end = _pilot_t_end(spec, spec.log_rates.astype(np.float32).astype(np.float64))
    ts = W.uniform_sample_grid(t_end, 9)
    obs_sp = [0, 1, 2]
    n = 512
    dl = W.seeded_dl_dobs(4, n, len(ts), len(obs_sp), scale=1.0 / n)
    snet, fw, orc, gev = _run_both(S, spec, n, t_end, ts, obs_sp, 6, dl=dl, T=0.5, max_steps=1 << 14, tpt=1)
    assert fw.run.variant == 1
    same = _compare_events(orc, fw, gev, t_end, spec.n_reactions, floor=0.99)
    _check_obs(spec, fw, orc, same, ts, np.asarray(obs_sp))
    agree = _bracket_agreement(orc, fw, np.asarray(ts), spec.n_reactions)
    same &= agree
    dl_g = dl.copy()
    dl_g[~same] = 0.0
    g = S.backward(fw, torch.tensor(dl_g, dtype=torch.float32, device="cuda"), 0.5).double().cpu().numpy()
    ref = orc.dtheta[same].sum(0)
    assert np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30) < GRAD_RTOL


@pytest.mark.parametrize("selector", ["gumbel", "soft"])
def test_bin_shards_reproduce_the_full_run(S, selector):
    """Trajectory ids are global: a run of ids [offset, offset + count) gives the same bin rows as the same
    rows of one run over all ids (the sharded multi-GPU path relies on it)."""
    net = W.ion_channel_coi()
    ts = W.uniform_sample_grid(8.0, 100)
    snet = S.Network(net)
    theta = torch.tensor(net.log_rates.astype(np.float32), device="cuda")
    kw = dict(readout="bin", max_steps=64, selector=selector, temperature=0.3 if selector == "soft" else None)
    full = S.forward(snet, theta, 3000, net.x0, 8.0, ts, [1], 8, **kw)
    part = S.forward(snet, theta, 1000, net.x0, 8.0, ts, [1], 8, traj_offset=1234, **kw)
    assert torch.equal(part.obs, full.obs[1234:2234])
    assert torch.equal(part.draws, full.draws[1234:2234])


@pytest.mark.parametrize("selector", ["gumbel", "soft"])
@pytest.mark.parametrize("record", [False, True])
@pytest.mark.parametrize("specialize", [True, False])
def test_bin_writes_every_bin_with_a_partial_last_warp(S, selector, record, specialize):
    """3,000 trajectories leave a last warp of 24 lanes; the warp-wide writes of the held bins must still
    cover every bin (the output starts as NaN); exact paths stay in the range of the open count (relaxed
    states of the soft forward can leave it)."""
    if selector == "soft" and not specialize:
        pytest.skip("the soft forward runs on the network-specialised kernels only")
    net = W.ion_channel_coi()
    ts = W.uniform_sample_grid(8.0, 100)
    snet = S.Network(net)
    theta = torch.tensor(net.log_rates.astype(np.float32), device="cuda")
    out = torch.full((3000, 100, 1), float("nan"), device="cuda")
    fw = S.forward(snet, theta, 3000, net.x0, 8.0, ts, [1], 8, readout="bin", max_steps=64, obs_out=out,
                   record=record, specialize=specialize, selector=selector,
                   temperature=0.3 if selector == "soft" else None)
    o = fw.obs.cpu().numpy()
    assert not np.isnan(o).any(), np.argwhere(np.isnan(o))[:5]
    if selector == "gumbel":
        assert o.min() >= 0.0 and o.max() <= 2.0


@pytest.mark.parametrize("n", [96, 100])
def test_bin_many_held_runs_overflow_the_run_buffer(S, n):
    """Immigration-death at low rates on a fine grid: each interval spans tens of bins, so a trajectory
    holds far more runs of whole bins than the per-thread buffer keeps; the runs past it are written by the
    thread itself. Bin averages and gradients against the oracle, full and partial last warp."""
    net = W.immigration_death(1.0, 0.1)
    ts = W.uniform_sample_grid(100.0, 5000)
    dl = W.seeded_dl_dobs(2, n, len(ts), 1, scale=1.0 / n)
    snet, fw, orc, gev = _run_both(S, net, n, 100.0, ts, [0], 12, dl=dl, T=0.5, max_steps=2048, K=64)
    assert np.all(fw.status.cpu().numpy() <= 1)
    same = _compare_events(orc, fw, gev, 100.0, net.n_reactions, floor=0.99)
    _check_obs(net, fw, orc, same, ts, np.array([0]))
    agree = _bracket_agreement(orc, fw, np.asarray(ts), net.n_reactions)
    same &= agree
    dl_g = dl.copy()
    dl_g[~same] = 0.0
    g = S.backward(fw, torch.tensor(dl_g, dtype=torch.float32, device="cuda"), 0.5).double().cpu().numpy()
    ref = orc.dtheta[same].sum(0)
    assert np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30) < GRAD_RTOL


def test_bin_without_samples(S):
    net = W.ion_channel_coi()
    snet = S.Network(net)
    theta = torch.tensor(net.log_rates.astype(np.float32), device="cuda")
    fw = S.forward(snet, theta, 64, net.x0, 8.0, np.zeros(0), [1], 0, readout="bin", record=True, max_steps=64)
    assert fw.obs.shape == (64, 0, 1) and torch.all(fw.status <= 1)
    g = S.backward(fw, torch.zeros(0, 1, device="cuda"), 0.5)
    assert torch.count_nonzero(g) == 0


WARP_CASES = {
    "ion_channel": lambda: (W.ion_channel_coi(), 8.0, W.uniform_sample_grid(8.0, 80), [1], 1024),
    "ragged_bins": lambda: (W.mixed_orders_toy(), 5.0, np.array([1e-3, 0.5, 0.5 + 1e-6, 0.75, 3.0, 4.999, 5.0]),
                            [0, 2], 333),
    "held_runs": lambda: (W.immigration_death(1.0, 0.1), 100.0, W.uniform_sample_grid(100.0, 3000), [0], 96),
    "random_160": lambda: (W.random_network(np.random.default_rng(31), n_species_range=(8, 16),
                                            n_reactions_range=(160, 160)), None, None, [0, 1, 2, 3], 256),
}


@pytest.mark.parametrize("shared", [False, True])
@pytest.mark.parametrize("case", sorted(WARP_CASES))
def test_bin_on_warp_kernels_matches_oracle(S, case, shared):
    """The bin readout on the warp-per-trajectory kernels (networks with hundreds of reactions): bin averages
    within the tolerance above on the trajectories whose events agree (long held runs written warp-wide
    included), and the straight-through gradient against the oracle's, with one upstream gradient per
    trajectory and with one shared by all (the prefix-sum path)."""
    net, t_end, ts, obs_sp, n = WARP_CASES[case]()
    if t_end is None:
        from test_gpu_warp import _pilot_t_end
        t_end = _pilot_t_end(net, net.log_rates.astype(np.float32).astype(np.float64))
        ts = W.uniform_sample_grid(t_end, 17)
    ts = np.asarray(ts)
    T = 0.4
    g1 = W.seeded_dl_dobs(7, 1, len(ts), len(obs_sp), scale=1.0 / n)
    dl = np.repeat(g1, n, axis=0) if shared else W.seeded_dl_dobs(7, n, len(ts), len(obs_sp), scale=1.0 / n)
    snet, fw, orc, gev = _run_both(S, net, n, t_end, ts, obs_sp, 21, dl=dl, T=T, max_steps=1 << 15, K=16, tpt=32)
    assert fw.run.variant == 32
    np.testing.assert_array_equal(fw.status.cpu().numpy(), orc.status)
    same = _compare_events(orc, fw, gev, t_end, net.n_reactions, floor=0.99)
    _check_obs(net, fw, orc, same, ts, np.asarray(obs_sp))
    agree = _bracket_agreement(orc, fw, ts, net.n_reactions)
    same &= agree
    if shared:
        # one upstream gradient for every trajectory: the oracle's sum over the agreeing ones
        assert same.all() or same.mean() > 0.98
        up = torch.tensor(g1[0], dtype=torch.float32, device="cuda")
        keep = same
    else:
        dl_g = dl.copy()
        dl_g[~same] = 0.0
        up = torch.tensor(dl_g, dtype=torch.float32, device="cuda")
        keep = same
    g = S.backward(fw, up, T).cpu().numpy().astype(np.float64)
    _, mism = fw.run.status_counts()
    assert mism == 0
    if shared and not same.all():
        pytest.skip("a trajectory disagrees; the shared upstream gradient cannot exclude it")
    ref = orc.dtheta[keep].sum(0)
    rel = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30)
    assert rel < GRAD_RTOL, (rel, g, ref)
