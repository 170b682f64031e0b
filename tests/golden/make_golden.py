"""Writes the stored expected values under tests/golden/ from the oracle's exact CME tools only.

    python tests/golden/make_golden.py

dimer_2a_b_cme.json: for 2A <-> B with a1 = k1 A (A - 1)/2, a2 = k2 B, k = (0.01, 0.1), A0 = 100
(the chain A + 2B = 100 has exactly 51 states, so Eq. 1 is solved with no truncation):
E[A](t_s) and Var[A](t_s) on t_s = s, s = 1..50, by the matrix exponential, and the stationary
mean and variance both from p Q = 0 and from detailed balance along B = 0..50.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import cme  # noqa: E402
import ssa_workloads as W  # noqa: E402


def dimer_cme():
    net = W.dimerization_2a_b(0.01, 0.1, 100)
    ts = W.uniform_sample_grid(50.0, 50)
    states, idx = cme.reachable_states(net, net.x0)
    Q = cme.generator(net, net.log_rates, states, idx)
    p0 = np.zeros(len(states))
    p0[idx[tuple(int(v) for v in net.x0)]] = 1.0
    P = cme.transient(Q, p0, ts)
    A = np.array([s[0] for s in states], dtype=np.float64)
    mean = P @ A
    var = P @ A ** 2 - mean ** 2
    ps = cme.stationary(Q)
    B = np.arange(51)
    Ab = 100 - 2 * B
    up = 0.01 * Ab * (Ab - 1) / 2.0
    down = 0.1 * B
    pdb = cme.detailed_balance_chain(up, down)
    # the transient ODE dp/dt = p Q also gives the gradient with respect to log k
    dmean = []
    for r in range(net.n_params):
        dQ = cme.generator_derivative(net, net.log_rates, states, idx, r)
        dP = cme.transient_gradient(Q, dQ, p0, ts)
        dmean.append((dP @ A).tolist())
    return {
        "network": "2A<->B, a1=k1*A*(A-1)/2, a2=k2*B, k1=0.01, k2=0.1, A0=100, B0=0",
        "cite": "arXiv 2602.19775 Eq. 1 (chemical master equation); Section 2 (homodimer propensity)",
        "n_states": len(states),
        "sample_times": ts.tolist(),
        "mean_A": mean.tolist(),
        "var_A": var.tolist(),
        "dmean_A_dlogk": dmean,
        "stationary_mean_A_generator": float(ps @ A),
        "stationary_var_A_generator": float(ps @ A ** 2 - (ps @ A) ** 2),
        "stationary_mean_A_detailed_balance": float(pdb @ Ab),
        "stationary_var_A_detailed_balance": float(pdb @ Ab ** 2 - (pdb @ Ab) ** 2),
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "dimer_2a_b_cme.json")
    with open(out, "w") as f:
        json.dump(dimer_cme(), f, indent=1)
    print("wrote", out)
