"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test ties the oracle to something other than itself:
* Philox4x32-10 words against cuRAND's host generator (an independent library implementation);
* the forward law against the exact chemical master equation (Eq. 1) of 2A <-> B (51 states),
  the Poisson law of immigration-death, and exact enumeration of short jump chains;
* the hand adjoint against float64 autograd of the literal straight-through graph (Eq. 5);
* the expected one-step straight-through gradient against a one-dimensional quadrature, and its
  T -> 0 limit against the exact derivative of the categorical probability (Section 3.3);
* invariants: a loss on a conserved quantity has zero gradient, and a rate shared by every
  reaction gets no gradient through the choice (softmax rows sum to one).
"""
import ctypes
import ctypes.util
import json
import os

import numpy as np
import pytest

import ssa_workloads as W
from ssa_workloads.configs import HOLD, LINEAR
from oracle import autodiff, cme, native, quadrature

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------------------------------------
# Philox
# ---------------------------------------------------------------------------------------------
def _curand_host():
    for name in ("libcurand.so.10", "libcurand.so", "/usr/local/cuda/lib64/libcurand.so.10"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not available")
    for seed in (0, 7, 0x123456789ABCDEF0, 2**64 - 1):
        g = ctypes.c_void_p()
        assert lib.curandCreateGeneratorHost(ctypes.byref(g), 161) == 0  # PHILOX4_32_10
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        nb = 2048
        ref = np.zeros(4 * nb, dtype=np.uint32)
        assert lib.curandGenerate(g, ref.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(4 * nb)) == 0
        lib.curandDestroyGenerator(g)
        # cuRAND's host generator lays block i of its output on counter (0, 0, i, 0)
        ctr = np.zeros((nb, 4), dtype=np.uint32)
        ctr[:, 2] = np.arange(nb)
        ours = native.philox_blocks(seed, ctr)
        np.testing.assert_array_equal(ours.reshape(-1), ref)


def test_uniform_mapping_is_open_interval_and_binary32_exact():
    u = np.concatenate([native.uniforms(5, traj, step, 9) for traj in range(50) for step in range(40)])
    assert np.all(u > 0.0) and np.all(u < 1.0)
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    # 23-bit grid offset by half a step
    m = u * 2.0 ** 23 - 0.5
    assert np.all(m == np.round(m))
    # roughly uniform
    assert abs(u.mean() - 0.5) < 0.01


# ---------------------------------------------------------------------------------------------
# Forward law
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("selector", ["gumbel", "direct"])
def test_dimer_2a_b_matches_exact_cme(selector):
    gold = json.load(open(os.path.join(GOLDEN, "dimer_2a_b_cme.json")))
    wl = W.config_c1()
    n = 65536
    r = native.run(wl.net, wl.log_rates, wl.x0, n, wl.t_end, wl.sample_times, wl.obs_species, 0, HOLD,
                   selector=selector)
    assert np.all(r.status == native.STATUS["OK"])
    A = r.obs[:, :, 0]
    B = r.obs[:, :, 1]
    np.testing.assert_array_equal(A + 2 * B, 100)  # conservation, exactly
    m = A.mean(0)
    se = A.std(0, ddof=1) / np.sqrt(n)
    z = (m - np.array(gold["mean_A"])) / se
    assert np.all(np.abs(z) < 3.0), z
    v = A.var(0, ddof=1)
    # standard error of a sample variance: sqrt((mu4 - var^2)/n)
    mu4 = ((A - m) ** 4).mean(0)
    se_v = np.sqrt(np.maximum(mu4 - v ** 2, 1e-12) / n)
    zv = (v - np.array(gold["var_A"])) / se_v
    # 50 sample variances are tested at once: 3.5 SE each keeps the family-wise false-alarm rate near 2%
    assert np.all(np.abs(zv) < 3.5), zv


def test_direct_method_first_choice_law():
    """One step of the direct method from a fixed state picks reaction j with probability a_j / a0
    (Section 2): chi-square of 100,000 first draws of the mixed-orders network."""
    net = W.mixed_orders_toy()
    x = net.x0.astype(np.float64)
    k = np.exp(net.log_rates[net.rate_index])
    h = np.array([1.0 if r1 < 0 else (x[r1] if r2 < 0 else (x[r1] * (x[r1] - 1) / 2 if r1 == r2 else x[r1] * x[r2]))
                  for r1, r2 in net.reactants])
    prob = k * h / np.sum(k * h)
    n = 100_000
    r = native.run(net, net.log_rates, net.x0, n, 1e9, np.zeros(0), np.array([0], np.int32), 3, HOLD,
                   max_steps=1, ev_cap=1, selector="direct")
    counts = np.bincount(r.events[:, 0], minlength=net.n_reactions)
    exp = n * prob
    use = exp > 5
    chi2 = np.sum((counts[use] - exp[use]) ** 2 / exp[use])
    dof = int(use.sum()) - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof), (chi2, dof, counts, exp)
    assert np.all(counts[prob == 0] == 0)


def test_dimer_2a_b_stationary_two_routes_agree():
    gold = json.load(open(os.path.join(GOLDEN, "dimer_2a_b_cme.json")))
    assert gold["n_states"] == 51
    assert abs(gold["stationary_mean_A_generator"] - gold["stationary_mean_A_detailed_balance"]) < 1e-9
    assert abs(gold["stationary_var_A_generator"] - gold["stationary_var_A_detailed_balance"]) < 1e-8
    assert abs(gold["mean_A"][-1] - gold["stationary_mean_A_generator"]) < 1e-3


def test_immigration_death_poisson_law():
    lam, mu = 10.0, 1.0
    net = W.immigration_death(lam, mu)
    ts = np.array([0.1, 0.5, 1.0, 2.0, 8.0])
    n = 40000
    r = native.run(net, net.log_rates, net.x0, n, 8.0, ts, np.array([0], np.int32), 3, HOLD)
    A = r.obs[:, :, 0]
    mean = cme.immigration_death_mean(lam, mu, ts)
    m = A.mean(0)
    se = np.sqrt(mean / n)          # Poisson: variance = mean
    assert np.all(np.abs((m - mean) / se) < 3.0)
    v = A.var(0, ddof=1)
    se_v = np.sqrt((mean + 2 * mean ** 2) / n)  # Poisson: mu4 - var^2 = lambda + 2 lambda^2
    assert np.all(np.abs((v - mean) / se_v) < 3.0)
    # the whole law at t = 8 (stationary to 3e-4): chi-square against Poisson(10)
    from scipy import stats
    counts = np.bincount(A[:, -1].astype(int), minlength=40)[:40]
    p = stats.poisson.pmf(np.arange(40), mean[-1])
    keep = p * n > 20
    chi2 = (((counts[keep] - n * p[keep]) ** 2) / (n * p[keep])).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-3


def test_jump_chain_enumeration_a_b_c():
    net = W.dimerization_a_b_c(k1=0.5, k2=0.7, xa=2, xb=2)
    n = 40000
    for n_jumps in (1, 2, 5, 10):
        law, mean_t = cme.enumerate_jump_chain(net, net.log_rates, net.x0, n_jumps)
        r = native.run(net, net.log_rates, net.x0, n, 1e9, np.zeros(0), np.array([0], np.int32), 9,
                       HOLD, max_steps=n_jumps, ev_cap=n_jumps)
        assert np.all(r.status == native.STATUS["STEP_CAP"])
        C = r.final_x[:, 2]
        for state, p in law.items():
            f = np.mean(C == state[2])
            se = np.sqrt(p * (1 - p) / n) + 1e-12
            assert abs(f - p) < 3.5 * se + 1e-12, (n_jumps, state, f, p)
        t_n = r.times[:, n_jumps - 1]
        se_t = t_n.std(ddof=1) / np.sqrt(n)
        assert abs(t_n.mean() - mean_t[-1]) < 3.0 * se_t


# ---------------------------------------------------------------------------------------------
# Backward
# ---------------------------------------------------------------------------------------------
def _autodiff_case(net, t_end, S, obs_sp, readout, T, seed, n, include_zero=True):
    ts = np.linspace(0.0, t_end, S) if include_zero else W.uniform_sample_grid(t_end, S)
    g = W.seeded_dl_dobs(seed + 1, n, S, len(obs_sp))
    r = native.run(net, net.log_rates, net.x0, n, t_end, ts, np.array(obs_sp, np.int32), seed,
                   readout, dl_dobs=g, temperature=T, ev_cap=5000)
    worst = 0.0
    for i in range(n):
        nd = int(r.draws[i])
        crossed = r.status[i] == native.STATUS["OK"]
        n_states = nd if crossed else nd + 1
        gt, obs = autodiff.st_gradient(net, net.log_rates, net.x0, r.events[i, :nd], n_states, crossed,
                                       seed, i, t_end, ts, obs_sp, readout, g[i], T)
        np.testing.assert_allclose(obs, r.obs[i], rtol=0, atol=1e-9)
        worst = max(worst, np.abs(gt - r.dtheta[i]).max() / max(np.abs(gt).max(), 1e-300))
    return worst


@pytest.mark.parametrize("readout", [HOLD, LINEAR])
def test_hand_adjoint_matches_autograd_mixed_orders(readout):
    net = W.mixed_orders_toy()
    assert _autodiff_case(net, 5.0, 7, [0, 1, 2], readout, 0.7, 11, 5) < 1e-10


@pytest.mark.parametrize("readout", [HOLD, LINEAR])
@pytest.mark.parametrize("T", [0.1, 1.0])
def test_hand_adjoint_matches_autograd_dimer(readout, T):
    net = W.dimerization_2a_b()
    assert _autodiff_case(net, 3.0, 5, [0, 1], readout, T, 21, 4, include_zero=False) < 1e-10


def test_hand_adjoint_matches_autograd_oscillator_short():
    net = W.vilar_oscillator()
    assert _autodiff_case(net, 0.05, 4, [6, 7, 8], LINEAR, 0.5, 4, 2) < 1e-10


def _branching_net(k1, k2):
    # S -> P1 (k1), S -> P2 (k2) with one S molecule: exactly one draw, then absorbing
    return W.network_from_reactions(["S", "P1", "P2"], [(["S"], ["P1"], "k1"), (["S"], ["P2"], "k2")],
                                    rates={"k1": k1, "k2": k2}, x0={"S": 1})


@pytest.mark.parametrize("T", [1.0, 0.5, 0.1])
def test_one_step_st_gradient_matches_quadrature(T):
    net = _branching_net(1.0, 0.5)
    n = 60000
    g = np.zeros((n, 1, 1))
    g[:, 0, 0] = 1.0  # L = P1 at t_end (HOLD): the straight-through derivative of y~_1
    r = native.run(net, net.log_rates, net.x0, n, 1e6, np.array([1e6]), np.array([1], np.int32), 13,
                   HOLD, dl_dobs=g, temperature=T)
    assert np.all(r.status == native.STATUS["ABSORBED"])
    d = r.dtheta[:, 0]
    np.testing.assert_allclose(r.dtheta[:, 1], -d, rtol=0, atol=1e-12)  # softmax rows sum to one
    expect = quadrature.expected_st_derivative(np.log(1.0 / 0.5), T)
    se = d.std(ddof=1) / np.sqrt(n)
    assert abs(d.mean() - expect) < 3.0 * se, (d.mean(), expect, se)


def test_one_step_st_gradient_low_temperature_limit_is_exact_derivative():
    lr = np.log(2.0)
    exact = quadrature.exact_choice_derivative(lr)
    assert abs(quadrature.expected_st_derivative(lr, 1e-3) - exact) < 1e-5
    assert abs(quadrature.expected_st_derivative(lr, 1.0) - exact) > 1e-2  # the bias at warm T


def test_conserved_quantity_loss_has_zero_gradient():
    net = W.dimerization_2a_b()
    ts = W.uniform_sample_grid(5.0, 10)
    n = 32
    for readout in (HOLD, LINEAR):
        g = np.zeros((n, 10, 2))
        g[:, :, 0] = 1.0
        g[:, :, 1] = 2.0  # L = sum_s A + 2B
        r = native.run(net, net.log_rates, net.x0, n, 5.0, ts, np.array([0, 1], np.int32), 2, readout,
                       dl_dobs=g, temperature=0.5)
        assert np.abs(r.dtheta).max() < 1e-12


def test_shared_global_rate_gets_no_choice_gradient():
    # every reaction uses one parameter; HOLD readout has no waiting-time path
    spec = W.network_from_reactions(["A", "B"], [(["A"], ["B"], "k"), (["B"], ["A"], "k"), ([], ["A"], "k")],
                                    rates={"k": 0.7}, x0={"A": 5, "B": 5})
    ts = W.uniform_sample_grid(3.0, 6)
    g = W.seeded_dl_dobs(4, 16, 6, 2)
    r = native.run(spec, spec.log_rates, spec.x0, 16, 3.0, ts, np.array([0, 1], np.int32), 1, HOLD,
                   dl_dobs=g, temperature=0.3)
    assert np.abs(r.dtheta).max() < 1e-10


# ---------------------------------------------------------------------------------------------
# Degenerate cases
# ---------------------------------------------------------------------------------------------
def test_degenerate_cases():
    net = W.dimerization_2a_b()
    ts = np.array([0.0, 1.0, 2.0])
    # empty batch
    r = native.run(net, net.log_rates, net.x0, 0, 2.0, ts, np.array([0], np.int32), 0, HOLD)
    assert r.obs.shape == (0, 3, 1)
    # t_end = 0: one crossing draw, the state holds at x0
    r = native.run(net, net.log_rates, net.x0, 4, 0.0, np.array([0.0]), np.array([0], np.int32), 0, LINEAR)
    assert np.all(r.draws == 1) and np.all(r.obs[:, 0, 0] == 100)
    # absorbing from the start: A = 1, B = 0 has a0 = 0
    r = native.run(net, net.log_rates, np.array([1, 0], np.int32), 3, 2.0, ts, np.array([0], np.int32), 0,
                   LINEAR)
    assert np.all(r.status == native.STATUS["ABSORBED"]) and np.all(r.draws == 0) and np.all(r.obs == 1)
    # step cap
    r = native.run(net, net.log_rates, net.x0, 3, 1e9, ts, np.array([0], np.int32), 0, HOLD, max_steps=7)
    assert np.all(r.status == native.STATUS["STEP_CAP"]) and np.all(r.draws == 7)
    # rejected inputs
    with pytest.raises(ValueError):
        native.run(net, net.log_rates, net.x0, 2, 1.0, np.array([0.5, 0.2]), np.array([0], np.int32), 0, HOLD)
    with pytest.raises(ValueError):
        native.run(net, net.log_rates, net.x0, 2, 1.0, np.array([2.0]), np.array([0], np.int32), 0, HOLD)
