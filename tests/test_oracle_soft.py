"""Pins of the oracle's soft forward (arXiv 2602.19775, Section 3.3, Eq. 4: the state moves by the expected
stoichiometry of the soft sample) and of the exact gradient of that relaxed model, against facts the
oracle does not compute itself: the T -> 0 and T -> infinity limits of the softmax, linear conservation
laws, central finite differences of the (deterministic, given its noise) soft path, and float64 autograd
of the relaxed graph."""
from __future__ import annotations

import numpy as np
import pytest

import ssa_workloads as W
from ssa_workloads.configs import HOLD, LINEAR
from oracle import autodiff, cme, native

BIN = native.BIN


def test_soft_forward_at_low_temperature_is_the_hard_path():
    """As T -> 0 the soft sample is one-hot on the Gumbel-max choice: where every key gap of a path exceeds
    1e-4, T = 1e-7 puts exp(-1000) on the other reactions and the soft path is the hard path exactly."""
    wl = W.config_c1()
    n = 512
    hard = native.run(wl.net, wl.log_rates, wl.x0, n, wl.t_end, wl.sample_times, wl.obs_species, 3, HOLD, ev_cap=4096)
    soft = native.run(wl.net, wl.log_rates, wl.x0, n, wl.t_end, wl.sample_times, wl.obs_species, 3, HOLD, ev_cap=4096,
                      selector="soft", temperature=1e-7)
    clear = np.array([np.nanmin(hard.margins[i, :hard.draws[i]]) > 1e-4 for i in range(n)])
    assert clear.mean() > 0.5
    np.testing.assert_array_equal(soft.events[clear], hard.events[clear])
    np.testing.assert_array_equal(soft.obs[clear], hard.obs[clear])


def test_soft_forward_at_high_temperature_takes_the_mean_update():
    """As T -> infinity the soft sample is uniform over the active reactions: X_1 = x0 + mean_j v_j."""
    net = W.mixed_orders_toy()
    V = net.stoich_dense()
    r = native.run(net, net.log_rates, net.x0, 8, 50.0, np.array([50.0]), np.array([0, 1, 2], np.int32), 1, HOLD,
                   selector="soft", temperature=1e12, max_steps=1)
    assert np.all(r.status == native.STATUS["STEP_CAP"])
    # reactions with a zero propensity at x0 (those consuming C, with C = 0) are not in the mean
    active = cme.propensities(net, net.log_rates, net.x0) > 0
    want = net.x0 + V[active].mean(0)
    np.testing.assert_allclose(r.obs[:, 0, :], np.broadcast_to(want, (8, 3)), rtol=0, atol=1e-9)


def test_soft_forward_keeps_linear_conservation_laws():
    """Every v_j of 2A <-> B keeps A + 2B, so every soft update (a convex combination of them) does too."""
    wl = W.config_c1()
    r = native.run(wl.net, wl.log_rates, wl.x0, 256, wl.t_end, wl.sample_times, np.array([0, 1], np.int32), 2,
                   LINEAR, selector="soft", temperature=0.7)
    np.testing.assert_allclose(r.obs[:, :, 0] + 2 * r.obs[:, :, 1], 100.0, rtol=0, atol=1e-9)
    assert np.any(np.abs(r.obs[:, :, 0] - np.round(r.obs[:, :, 0])) > 1e-3)  # the states are relaxed


@pytest.mark.parametrize("readout", [LINEAR, BIN])
def test_soft_gradient_matches_finite_differences(readout):
    """The soft path is a smooth function of theta for fixed noise (until a draw count or a bracket changes),
    so its exact gradient is the limit of central differences."""
    net = W.mixed_orders_toy()
    t_end, n, T, h = 3.0, 24, 0.8, 1e-6
    ts = W.uniform_sample_grid(t_end, 6)
    obs_sp = np.array([0, 1, 2], np.int32)
    g = W.seeded_dl_dobs(7, n, len(ts), 3)
    base = native.run(net, net.log_rates, net.x0, n, t_end, ts, obs_sp, 5, readout, selector="soft", temperature=T,
                      dl_dobs=g, ev_cap=2000)
    fd = np.zeros((n, net.n_params))
    ok = np.ones(n, bool)
    for r in range(net.n_params):
        th_p, th_m = net.log_rates.copy(), net.log_rates.copy()
        th_p[r] += h
        th_m[r] -= h
        rp = native.run(net, th_p, net.x0, n, t_end, ts, obs_sp, 5, readout, selector="soft", temperature=T, ev_cap=2000)
        rm = native.run(net, th_m, net.x0, n, t_end, ts, obs_sp, 5, readout, selector="soft", temperature=T, ev_cap=2000)
        ok &= (rp.draws == base.draws) & (rm.draws == base.draws)
        fd[:, r] = ((rp.obs - rm.obs) * g).sum((1, 2)) / (2 * h)
    assert ok.mean() > 0.8
    err = np.abs(fd[ok] - base.dtheta[ok]).max() / np.abs(base.dtheta[ok]).max()
    assert err < 1e-5, err


@pytest.mark.parametrize("case", ["mixed_hold", "mixed_linear_hot", "dimer_bin", "ion_bin"])
def test_soft_hand_adjoint_matches_autograd(case):
    if case.startswith("mixed"):
        net, t_end, S, obs_sp = W.mixed_orders_toy(), 4.0, 7, [0, 1, 2]
        readout = HOLD if case == "mixed_hold" else LINEAR
        T = 0.6 if case == "mixed_hold" else 3.0  # hot: relaxed states leave the integers, clipping engages
    elif case == "dimer_bin":
        net, t_end, S, obs_sp, readout, T = W.dimerization_2a_b(), 3.0, 5, [0, 1], BIN, 0.4
    else:
        net, t_end, S, obs_sp, readout, T = W.ion_channel_coi(), 8.0, 12, [1], BIN, 0.5
    ts = W.uniform_sample_grid(t_end, S)
    n, seed = 4, 17
    g = W.seeded_dl_dobs(seed + 1, n, S, len(obs_sp))
    r = native.run(net, net.log_rates, net.x0, n, t_end, ts, np.array(obs_sp, np.int32), seed, readout, dl_dobs=g,
                   temperature=T, ev_cap=5000, selector="soft")
    for i in range(n):
        nd = int(r.draws[i])
        crossed = r.status[i] == native.STATUS["OK"]
        n_states = nd if crossed else nd + 1
        gt, obs = autodiff.st_gradient(net, net.log_rates, net.x0, r.events[i, :nd], n_states, crossed, seed, i,
                                       t_end, ts, obs_sp, readout, g[i], T, soft=True)
        np.testing.assert_allclose(obs, r.obs[i], rtol=1e-11, atol=1e-9)
        np.testing.assert_allclose(gt, r.dtheta[i], rtol=1e-9, atol=1e-12 * np.abs(gt).max())


def test_soft_rejects_missing_temperature():
    wl = W.config_c1()
    with pytest.raises(ValueError):
        native.run(wl.net, wl.log_rates, wl.x0, 2, 1.0, np.array([1.0]), np.array([0], np.int32), 0, HOLD,
                   selector="soft", temperature=0.0)
