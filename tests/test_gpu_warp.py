"""GPU parity of the warp-per-trajectory kernels (networks with many reactions) against the FP64
oracle: event sequences under the margin rule, observables, and straight-through gradients on
trajectories whose events and sample brackets agree."""
import numpy as np
import pytest
import torch

import ssa_workloads as W
from ssa_workloads.configs import HOLD, LINEAR
from oracle import native

from test_gpu_parity import (GRAD_RTOL, _bracket_agreement, _clock_tol, _compare_events,
                              _oracle_brackets, _theta32)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2602_19775_gb300 import ssa
    ssa._lib.lib()
    return ssa


def _pilot_t_end(net, theta64, target_draws=150, seed=99):
    """Horizon giving about `target_draws` draws per trajectory (oracle pilot on 16 trajectories)."""
    t_end = 1.0
    for _ in range(30):
        o = native.run(net, theta64, net.x0, 16, t_end, np.zeros(0), np.array([0], np.int32), seed, HOLD,
                       max_steps=20 * target_draws)
        m = o.draws.mean()
        if 0.5 * target_draws <= m <= 2 * target_draws and np.all(o.status <= 2):
            return t_end
        t_end *= (target_draws / max(m, 1.0)) ** 0.9 if m > 0 else 4.0
    return t_end


def _parity(S, net, theta, n, t_end, S_samples, obs_sp, seed, readout, T, tpt, max_steps=4096, dl_seed=7):
    t32, t64 = _theta32(theta)
    ts = W.uniform_sample_grid(t_end, S_samples)
    dl = W.seeded_dl_dobs(dl_seed, n, S_samples, len(obs_sp), scale=1.0 / n)
    snet = S.Network(net)
    fw = S.forward(snet, torch.tensor(t32, device="cuda"), n, net.x0, t_end, ts, obs_sp, seed,
                   readout="hold" if readout == HOLD else "linear", record=True, max_steps=max_steps,
                   threads_per_traj=tpt)
    orc = native.run(net, t64, net.x0, n, t_end, ts, obs_sp, seed, readout, max_steps=max_steps, dl_dobs=dl,
                     temperature=T, ev_cap=max_steps)
    gst = fw.status.cpu().numpy()
    np.testing.assert_array_equal(gst, orc.status)
    same = _compare_events(orc, fw, fw.run.events(max_steps).cpu().numpy(), t_end, net.n_reactions, floor=0.99)
    agree = _bracket_agreement(orc, fw, ts, net.n_reactions)
    use = same & agree
    obs = fw.obs.double().cpu().numpy()
    if readout == HOLD:
        assert np.all(obs[use] == orc.obs[use])
    else:
        # alpha = (t_s - t_k)/tau_k moves by at most clock_tol/tau_k; |X_{k+1} - X_k| <= max |v|
        ob = _oracle_brackets(orc, ts)
        vmax = np.abs(net.stoich_delta).max()
        for i in np.nonzero(use)[0]:
            t = np.concatenate([[0.0], orc.times[i, :orc.draws[i]]])
            k = ob[i]
            tau = t[np.minimum(k + 1, len(t) - 1)] - t[k]
            tol = vmax * _clock_tol(net.n_reactions, ts) / np.maximum(tau, 1e-300) + 1e-6 * np.abs(orc.obs[i]).max(1)
            assert np.all(np.abs(obs[i] - orc.obs[i]).max(1) <= tol), i
    dl_g = dl.copy()
    dl_g[~use] = 0
    g = S.backward(fw, torch.tensor(dl_g, dtype=torch.float32, device="cuda"), T).cpu().numpy().astype(np.float64)
    ref = orc.dtheta[use].sum(0)
    _, mism = fw.run.status_counts()
    assert mism == 0
    rel = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30)
    assert rel < GRAD_RTOL, (rel, np.abs(g - ref).max(), np.abs(ref).max())
    return rel, use.mean()


@pytest.mark.parametrize("readout", [HOLD, LINEAR])
def test_warp_kernel_on_dimer(S, readout):
    wl = W.config_c2(n_traj=2048)
    _parity(S, wl.net, wl.log_rates, 2048, 50.0, 50, np.array([0, 1], np.int32), 3, readout, 0.5, tpt=32)


def test_warp_kernel_on_oscillator(S):
    net = W.vilar_oscillator()
    _parity(S, net, net.log_rates, 256, 1.0, 20, np.array([6, 7, 8], np.int32), 5, LINEAR, 0.3, tpt=32,
            max_steps=1 << 14)


def test_warp_kernel_on_mixed_orders(S):
    net = W.mixed_orders_toy()
    _parity(S, net, net.log_rates, 1000, 6.0, 11, np.array([0, 1, 2], np.int32), 9, HOLD, 0.5, tpt=32)


@pytest.mark.parametrize("seed", [3, 10, 14])
def test_random_networks_with_hundreds_of_reactions(S, seed):
    rng = np.random.default_rng(seed)
    net = W.random_network(rng, n_species_range=(8, 64), n_reactions_range=(100, 512))
    theta = net.log_rates.astype(np.float32).astype(np.float64)
    t_end = _pilot_t_end(net, theta)
    obs = np.arange(min(4, net.n_species), dtype=np.int32)
    for readout in (HOLD, LINEAR):
        _parity(S, net, net.log_rates, 256, t_end, 12, obs, seed, readout, 1.0, tpt=0)


def test_thread_and_warp_variants_agree_with_each_other(S):
    rng = np.random.default_rng(5)
    net = W.random_network(rng, n_species_range=(6, 12), n_reactions_range=(20, 40))
    theta = net.log_rates.astype(np.float32).astype(np.float64)
    t_end = _pilot_t_end(net, theta)
    snet = S.Network(net)
    th = torch.tensor(net.log_rates.astype(np.float32), device="cuda")
    ts = W.uniform_sample_grid(t_end, 8)
    a = S.forward(snet, th, 1024, net.x0, t_end, ts, [0, 1], 4, record=True, threads_per_traj=1)
    b = S.forward(snet, th, 1024, net.x0, t_end, ts, [0, 1], 4, record=True, threads_per_traj=32)
    ea, eb = a.run.events(4096).cpu().numpy(), b.run.events(4096).cpu().numpy()
    # the two variants sum a0 and reduce the race in different orders: they may part only at near-ties
    assert np.mean(np.all(ea == eb, axis=1)) > 0.99


@pytest.mark.parametrize("M", [9, 10, 11])
def test_thread_kernel_with_nine_to_eleven_reactions(S, M):
    # the unrolled thread kernels evaluate 16 reactions here: the padded entries must be inert
    net = W.random_network(np.random.default_rng(100 + M), n_species_range=(3, 8), n_reactions_range=(M, M))
    theta = net.log_rates.astype(np.float32).astype(np.float64)
    t_end = _pilot_t_end(net, theta)
    _parity(S, net, net.log_rates, 512, t_end, 8, np.array([0, 1], np.int32), M, LINEAR, 0.5, tpt=1)
