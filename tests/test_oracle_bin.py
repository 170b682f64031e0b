"""Pins of the oracle's exact bin-averaged readout (arXiv 2602.19775, Section 4.4) and of the
straight-through gradient through it, against facts the oracle does not compute itself: closed-form
means, the chemical master equation (Eq. 1) integrated over each bin, a midpoint Riemann sum of the
same path, a conserved quantity, the pathwise derivative of a one-reaction chain, and float64
autograd of the literal graph.

Bins are (t_{s-1}, t_s] with t_{-1} = 0: the sample times are the bins' right edges.
"""
from __future__ import annotations

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import ssa_workloads as W
from ssa_workloads.configs import HOLD
from ssa_workloads.networks import network_from_reactions
from oracle import autodiff, cme, native

BIN = native.BIN


def _lo(edges):
    return np.concatenate([[0.0], edges[:-1]])


def test_bin_average_helper_matches_quadrature():
    """transient_bin_average (Van Loan block exponential) against adaptive quadrature of p(t)."""
    rng = np.random.default_rng(7)
    Q = rng.uniform(0.1, 2.0, (4, 4))
    np.fill_diagonal(Q, 0.0)
    Q -= np.diag(Q.sum(1))
    p0 = np.array([1.0, 0.0, 0.0, 0.0])
    edges = np.array([0.3, 0.35, 1.0, 2.5])
    got = cme.transient_bin_average(Q, p0, edges)
    for s, (lo, b) in enumerate(zip(_lo(edges), edges)):
        val, _ = scipy.integrate.quad_vec(lambda t: p0 @ scipy.linalg.expm(Q * t), lo, b, epsabs=1e-13,
                                          epsrel=1e-12)
        np.testing.assert_allclose(got[s], val / (b - lo), rtol=0, atol=1e-10)


def _z_means(obs, exact):
    n = obs.shape[0]
    se = obs.std(0, ddof=1) / np.sqrt(n)
    return (obs.mean(0) - exact) / np.maximum(se, 1e-300)


def test_pure_death_bin_means_and_pathwise_gradient():
    """A -> 0 from x0: E[X(t)] = x0 exp(-k t), so the bin mean is x0 (e^{-k lo} - e^{-k b}) / (k D).
    With one reaction the soft sample is identically 1, so the straight-through gradient is the
    pathwise derivative of the event times (tau = E/(k X)); the bin average is Lipschitz in the
    times, hence its expectation is d E[L]/d log k exactly."""
    k, x0 = 0.7, 20
    net = network_from_reactions(["A"], [(["A"], [], "k")], rates={"k": k}, x0={"A": x0})
    edges = np.array([0.2, 0.5, 1.0, 1.7, 3.0, 5.0])
    lo, D = _lo(edges), edges - _lo(edges)
    n = 40000
    c = np.random.default_rng(3).normal(size=len(edges))
    g = np.ascontiguousarray(np.broadcast_to(c[None, :, None], (n, len(edges), 1)))
    r = native.run(net, net.log_rates, net.x0, n, 5.0, edges, np.array([0], np.int32), 9, BIN, dl_dobs=g,
                   temperature=0.5)
    f = (np.exp(-k * lo) - np.exp(-k * edges)) / k
    mean = x0 * f / D
    z = _z_means(r.obs[:, :, 0], mean)
    assert np.all(np.abs(z) < 3.5), z
    df_dk = (-lo * np.exp(-k * lo) + edges * np.exp(-k * edges)) / k - f / k
    exact = float((c * x0 * k * df_dk / D).sum())
    st = r.dtheta[:, 0]
    zg = (st.mean() - exact) / (st.std(ddof=1) / np.sqrt(n))
    assert abs(zg) < 3.5, (st.mean(), exact, zg)


def test_immigration_death_bin_means_closed_form():
    """0 -> A (lam), A -> 0 (mu) from 0: E[X(t)] = lam/mu (1 - e^{-mu t}), integrated over each bin."""
    lam, mu = 10.0, 1.0
    net = W.immigration_death(lam, mu)
    edges = W.uniform_sample_grid(6.0, 30)
    lo, D = _lo(edges), edges - _lo(edges)
    mean = lam / mu * (1.0 - (np.exp(-mu * lo) - np.exp(-mu * edges)) / (mu * D))
    r = native.run(net, net.log_rates, net.x0, 40000, 6.0, edges, np.array([0], np.int32), 4, BIN)
    z = _z_means(r.obs[:, :, 0], mean)
    assert np.all(np.abs(z) < 3.5), z


@pytest.mark.parametrize("which", ["ion_channel", "dimer"])
def test_bin_means_match_cme(which):
    """Ensemble means of the bin averages against the CME law averaged over each bin (Eq. 1)."""
    if which == "ion_channel":
        net = W.ion_channel_coi()
        edges, obs_sp, t_end, n = W.uniform_sample_grid(8.0, 40), 1, 8.0, 40000
    else:
        net = W.dimerization_2a_b(0.01, 0.1, 40)
        edges, obs_sp, t_end, n = W.uniform_sample_grid(20.0, 40), 0, 20.0, 20000
    states, index = cme.reachable_states(net, net.x0)
    Q = cme.generator(net, net.log_rates, states, index)
    p0 = np.zeros(len(states))
    p0[index[tuple(int(v) for v in net.x0)]] = 1.0
    pbar = cme.transient_bin_average(Q, p0, edges)
    mean = pbar @ np.array([x[obs_sp] for x in states], dtype=np.float64)
    r = native.run(net, net.log_rates, net.x0, n, t_end, edges, np.array([obs_sp], np.int32), 5, BIN)
    z = _z_means(r.obs[:, :, 0], mean)
    # 40 correlated bins at 3.5 SE each: family-wise false-alarm rate under 2%
    assert np.all(np.abs(z) < 3.5), z


def test_bin_average_matches_midpoint_riemann_sum_of_the_same_path():
    """The same trajectories (same seed) sampled with HOLD at the midpoints of a fine grid: the
    midpoint rule of a step function errs by at most |jump| h / 2 per jump inside the bin."""
    net = W.mixed_orders_toy()
    edges = np.array([0.5, 1.0, 2.25, 3.0, 5.0])
    n, h = 6, 1e-3
    obs_sp = np.array([0, 1, 2], np.int32)
    rb = native.run(net, net.log_rates, net.x0, n, 5.0, edges, obs_sp, 13, BIN, ev_cap=4000)
    grid = np.arange(0.0, 5.0, h) + h / 2
    rh = native.run(net, net.log_rates, net.x0, n, 5.0, grid, obs_sp, 13, HOLD)
    for s, (lo, b) in enumerate(zip(_lo(edges), edges)):
        m = (grid > lo) & (grid < b)
        riemann = rh.obs[:, m, :].mean(1)
        t_ev = rb.times
        for i in range(n):
            jumps = np.sum((t_ev[i] > lo) & (t_ev[i] <= b))
            bound = (jumps * 2 * h / 2 + 1e-12) / (b - lo) + 1e-9
            assert np.all(np.abs(rb.obs[i, s] - riemann[i]) <= bound), (s, i, rb.obs[i, s], riemann[i])


def test_conserved_quantity_has_zero_bin_gradient():
    """A + 2B is constant on every path of 2A <-> B, so its bin averages are constant and a loss
    on them has zero gradient: choice, state and time terms of the adjoint must cancel."""
    net = W.dimerization_2a_b()
    edges = W.uniform_sample_grid(5.0, 10)
    n = 64
    c = np.random.default_rng(1).normal(size=len(edges))
    g = np.zeros((n, len(edges), 2))
    g[:, :, 0] = c
    g[:, :, 1] = 2 * c
    r = native.run(net, net.log_rates, net.x0, n, 5.0, edges, np.array([0, 1], np.int32), 2, BIN, dl_dobs=g,
                   temperature=0.3)
    np.testing.assert_allclose(r.obs[:, :, 0] + 2 * r.obs[:, :, 1], 100.0, rtol=0, atol=1e-11)
    # the per-trajectory terms are O(1e3); they cancel to rounding
    assert np.abs(r.dtheta).max() < 1e-8, np.abs(r.dtheta).max()


def _autodiff_bin(net, t_end, S, obs_sp, T, seed, n):
    ts = W.uniform_sample_grid(t_end, S)
    g = W.seeded_dl_dobs(seed + 1, n, S, len(obs_sp))
    r = native.run(net, net.log_rates, net.x0, n, t_end, ts, np.array(obs_sp, np.int32), seed, BIN, dl_dobs=g,
                   temperature=T, ev_cap=5000)
    worst = 0.0
    for i in range(n):
        nd = int(r.draws[i])
        crossed = r.status[i] == native.STATUS["OK"]
        n_states = nd if crossed else nd + 1
        gt, obs = autodiff.st_gradient(net, net.log_rates, net.x0, r.events[i, :nd], n_states, crossed, seed, i,
                                       t_end, ts, obs_sp, BIN, g[i], T)
        np.testing.assert_allclose(obs, r.obs[i], rtol=0, atol=1e-9)
        worst = max(worst, np.abs(gt - r.dtheta[i]).max() / max(np.abs(gt).max(), 1e-300))
    return worst


@pytest.mark.parametrize("case", ["mixed_orders", "dimer_T0.1", "dimer_T1", "ion_channel", "oscillator"])
def test_bin_hand_adjoint_matches_autograd(case):
    if case == "mixed_orders":
        assert _autodiff_bin(W.mixed_orders_toy(), 5.0, 7, [0, 1, 2], 0.7, 11, 5) < 1e-10
    elif case.startswith("dimer"):
        T = 0.1 if case.endswith("0.1") else 1.0
        assert _autodiff_bin(W.dimerization_2a_b(), 3.0, 5, [0, 1], T, 21, 4) < 1e-10
    elif case == "ion_channel":
        assert _autodiff_bin(W.ion_channel_coi(), 8.0, 16, [1], 0.5, 31, 8) < 1e-10
    else:
        assert _autodiff_bin(W.vilar_oscillator(), 0.2, 6, [4, 6, 7], 0.5, 41, 2) < 1e-9


def test_bin_degenerate_cases():
    net = W.dimerization_2a_b()
    edges = np.array([0.5, 1.0, 2.0])
    g = np.ones((3, 3, 1))
    # absorbing from the start: the path is constant, every bin holds it, no gradient
    r = native.run(net, net.log_rates, np.array([1, 0], np.int32), 3, 2.0, edges, np.array([0], np.int32), 0, BIN,
                   dl_dobs=g, temperature=0.5)
    assert np.all(r.obs == 1.0) and np.all(r.dtheta == 0.0)
    # all channels inactivated: nothing is open in any bin
    ion = W.ion_channel_coi()
    r = native.run(ion, ion.log_rates, np.array([0, 0, 2], np.int32), 2, 2.0, edges, np.array([1], np.int32), 0,
                   BIN)
    assert np.all(r.obs == 0.0)
    # one bin over the whole horizon of a stopped path: the time-weighted mean of the visited states
    r = native.run(net, net.log_rates, net.x0, 4, 2.0, np.array([2.0]), np.array([0], np.int32), 6, BIN,
                   max_steps=3, ev_cap=8)
    assert np.all(r.status == native.STATUS["STEP_CAP"])
    for i in range(4):
        t = np.concatenate([[0.0], r.times[i, :3], [2.0]])
        xs = [100.0]  # reaction 0 is 2A -> B, reaction 1 is B -> 2A
        for j in r.events[i, :3]:
            xs.append(xs[-1] + (-2.0 if j == 0 else 2.0))
        want = sum(xs[q] * (t[q + 1] - t[q]) for q in range(4)) / 2.0
        assert abs(r.obs[i, 0, 0] - want) < 1e-12
    # rejected bins: t_0 = 0 (empty first bin) and repeated edges
    with pytest.raises(ValueError):
        native.run(net, net.log_rates, net.x0, 2, 1.0, np.array([0.0, 0.5]), np.array([0], np.int32), 0, BIN)
    with pytest.raises(ValueError):
        native.run(net, net.log_rates, net.x0, 2, 1.0, np.array([0.5, 0.5]), np.array([0], np.int32), 0, BIN)
