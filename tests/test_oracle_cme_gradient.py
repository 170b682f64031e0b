"""Pins of the oracle's exact CME gradient (`oracle.cme.transient_gradient`, Van Loan's block exponential of
[[Q, dQ], [0, Q]]), which serves as the exact reference for the straight-through estimator's bias.

* Immigration-death 0 -> A (lam), A -> 0 (mu A) from A = 0: E[A](t) = lam/mu (1 - e^{-mu t}), so
  d/dlog lam = E[A](t) and d/dlog mu = -lam/mu (1 - e^{-mu t}) + lam t e^{-mu t} (closed forms). The chain is
  truncated far in the tail (Poisson mean 5, 80 states) and its generator is written out here by hand.
* 2A <-> B (a1 = k1 A (A - 1)/2, a2 = k2 B, 51 states): the block exponential equals central finite
  differences of `cme.transient` in log k, at the true rates and at the evaluation point of the gradient
  workload, and the stored `dmean_A_dlogk` (tests/golden/dimer_2a_b_cme.json) equals a recomputation.
"""
import json
import os

import numpy as np

import ssa_workloads as W
from oracle import cme

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _birth_death(lam, mu, K):
    Q = np.zeros((K + 1, K + 1))
    dlam = np.zeros_like(Q)
    dmu = np.zeros_like(Q)
    for x in range(K + 1):
        if x < K:
            Q[x, x + 1] += lam
            Q[x, x] -= lam
            dlam[x, x + 1] += lam
            dlam[x, x] -= lam
        if x > 0:
            Q[x, x - 1] += mu * x
            Q[x, x] -= mu * x
            dmu[x, x - 1] += mu * x
            dmu[x, x] -= mu * x
    return Q, dlam, dmu


def test_transient_gradient_matches_immigration_death_closed_form():
    lam, mu, K = 5.0, 1.0, 80
    ts = np.array([0.1, 0.5, 1.0, 2.0, 5.0])
    Q, dlam, dmu = _birth_death(lam, mu, K)
    p0 = np.zeros(K + 1)
    p0[0] = 1.0
    A = np.arange(K + 1, dtype=np.float64)
    mean = cme.transient(Q, p0, ts) @ A
    np.testing.assert_allclose(mean, cme.immigration_death_mean(lam, mu, ts), rtol=1e-12)
    g_lam = cme.transient_gradient(Q, dlam, p0, ts) @ A
    g_mu = cme.transient_gradient(Q, dmu, p0, ts) @ A
    np.testing.assert_allclose(g_lam, lam / mu * (1.0 - np.exp(-mu * ts)), rtol=1e-10)
    np.testing.assert_allclose(g_mu, -lam / mu * (1.0 - np.exp(-mu * ts)) + lam * ts * np.exp(-mu * ts), rtol=1e-9)
    # probability is conserved: the gradient of the total mass is zero
    np.testing.assert_allclose(cme.transient_gradient(Q, dmu, p0, ts).sum(1), 0.0, atol=1e-12)


def _dimer_mean_and_gradient(theta):
    net = W.dimerization_2a_b(0.01, 0.1, 100)
    ts = W.uniform_sample_grid(50.0, 50)
    states, idx = cme.reachable_states(net, net.x0)
    p0 = np.zeros(len(states))
    p0[idx[tuple(int(v) for v in net.x0)]] = 1.0
    A = np.array([s[0] for s in states], dtype=np.float64)
    Q = cme.generator(net, theta, states, idx)
    mean = cme.transient(Q, p0, ts) @ A
    grad = np.stack([cme.transient_gradient(Q, cme.generator_derivative(net, theta, states, idx, r), p0, ts) @ A
                     for r in range(net.n_params)])
    return net, states, idx, p0, A, ts, mean, grad


def test_dimer_transient_gradient_matches_finite_differences():
    h = 1e-5
    for theta in (np.log([0.01, 0.1]), np.log([0.02, 0.05])):
        net, states, idx, p0, A, ts, mean, grad = _dimer_mean_and_gradient(theta)
        for r in range(2):
            tp, tm = theta.copy(), theta.copy()
            tp[r] += h
            tm[r] -= h
            mp = cme.transient(cme.generator(net, tp, states, idx), p0, ts) @ A
            mm = cme.transient(cme.generator(net, tm, states, idx), p0, ts) @ A
            fd = (mp - mm) / (2 * h)
            np.testing.assert_allclose(grad[r], fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max())
        # A + 2B = 100 is conserved, and dimerisation lowers A: d E[A]/d log k1 < 0 < d E[A]/d log k2
        assert np.all(grad[0] < 0) and np.all(grad[1] > 0)


def test_stored_cme_gradient_equals_recomputation():
    gold = json.load(open(os.path.join(GOLDEN, "dimer_2a_b_cme.json")))
    _, _, _, _, _, ts, mean, grad = _dimer_mean_and_gradient(np.log([0.01, 0.1]))
    np.testing.assert_allclose(gold["sample_times"], ts, rtol=0, atol=0)
    np.testing.assert_allclose(gold["mean_A"], mean, rtol=1e-12)
    np.testing.assert_allclose(np.array(gold["dmean_A_dlogk"]), grad, rtol=1e-10, atol=1e-12)
