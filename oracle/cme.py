"""Chemical master equation tools (arXiv 2602.19775, Section 2, Eq. 1).  Test infrastructure.

For a network whose reachable state set is finite, Eq. 1 is the linear ODE dp/dt = p Q with the
generator Q[x, x + v_j] += a_j(x), Q[x, x] = -a0(x). These functions build Q from the mass-action
propensities of Section 2, and give exact laws against which simulations are checked:

* ``transient``  p(t) = p(0) expm(Q t)   (scipy.linalg.expm; not an eigendecomposition, which
                 is ill-conditioned for these chains)
* ``stationary`` the probability vector with p Q = 0
* ``detailed_balance_chain`` the stationary law of a one-dimensional birth-death chain from
                 the ratio of its up and down rates
* ``immigration_death_mean`` the Poisson mean lam/mu (1 - exp(-mu t)) of 0 -> A, A -> 0 from A = 0
* ``enumerate_jump_chain``  the exact law of X_n after n jumps, P(path) = prod a_j/a0, and the
                 exact E[t_n] = E[sum_k 1/a0(X_k)]
* ``transient_gradient`` d p(t)/d log k_r via expm of [[Q, dQ], [0, Q]] (Van Loan's block form)
* ``transient_bin_average`` the average of p(t) over each bin, via expm of [[Q, I], [0, 0]]
"""
from __future__ import annotations

from collections import deque

import numpy as np
import scipy.linalg


def _h(reactants, x):
    r = [s for s in reactants if s >= 0]
    if len(r) == 0:
        return 1.0
    if len(r) == 1:
        return float(x[r[0]])
    if r[0] == r[1]:
        return float(x[r[0]]) * (float(x[r[0]]) - 1.0) / 2.0
    return float(x[r[0]]) * float(x[r[1]])


def propensities(net, log_rates, x):
    k = np.exp(np.asarray(log_rates, dtype=np.float64))[net.rate_index]
    return np.array([k[j] * _h(net.reactants[j], x) for j in range(net.n_reactions)])


def reachable_states(net, x0, max_states: int = 200000):
    """Breadth-first enumeration of the states reachable from x0 through reactions with a > 0
    (for any positive rates)."""
    V = net.stoich_dense()
    x0 = tuple(int(v) for v in x0)
    index = {x0: 0}
    order = [x0]
    q = deque([x0])
    ones = np.zeros(net.n_params)
    while q:
        x = q.popleft()
        a = propensities(net, ones, x)
        for j in range(net.n_reactions):
            if a[j] > 0:
                y = tuple(int(v) for v in np.asarray(x) + V[j])
                if min(y) < 0:
                    continue
                if y not in index:
                    if len(order) >= max_states:
                        raise ValueError("state space larger than max_states")
                    index[y] = len(order)
                    order.append(y)
                    q.append(y)
    return order, index


def generator(net, log_rates, states, index):
    """Q of Eq. 1 on the given closed state list; rows sum to zero."""
    V = net.stoich_dense()
    n = len(states)
    Q = np.zeros((n, n))
    for xi, x in enumerate(states):
        a = propensities(net, log_rates, x)
        for j in range(net.n_reactions):
            if a[j] > 0:
                y = tuple(int(v) for v in np.asarray(x) + V[j])
                Q[xi, index[y]] += a[j]
                Q[xi, xi] -= a[j]
    return Q


def generator_derivative(net, log_rates, states, index, r: int):
    """dQ/d log k_r: reactions using parameter r contribute a_j (since d a_j/d log k = a_j)."""
    V = net.stoich_dense()
    n = len(states)
    D = np.zeros((n, n))
    for xi, x in enumerate(states):
        a = propensities(net, log_rates, x)
        for j in range(net.n_reactions):
            if a[j] > 0 and net.rate_index[j] == r:
                y = tuple(int(v) for v in np.asarray(x) + V[j])
                D[xi, index[y]] += a[j]
                D[xi, xi] -= a[j]
    return D


def transient(Q, p0, times):
    """p(t) for each t (rows), by the matrix exponential."""
    return np.stack([p0 @ scipy.linalg.expm(Q * t) for t in times])


def transient_gradient(Q, dQ, p0, times):
    """d p(t)/d theta for a generator derivative dQ, from expm([[Q, dQ], [0, Q]] t)."""
    n = Q.shape[0]
    B = np.zeros((2 * n, 2 * n))
    B[:n, :n] = Q
    B[:n, n:] = dQ
    B[n:, n:] = Q
    out = []
    for t in times:
        E = scipy.linalg.expm(B * t)
        out.append(p0 @ E[:n, n:])
    return np.stack(out)


def transient_bin_average(Q, p0, edges):
    """(1/D_s) int over (b_{s-1}, b_s] of p(t) dt for the bins whose right edges are `edges` (b_{-1} = 0,
    D_s = b_s - b_{s-1} > 0): p(b_{s-1}) times the top-right block of expm([[Q, I], [0, 0]] D_s), which is
    int_0^D expm(Q u) du (Van Loan's block form), divided by D_s. These are the exact means of the
    bin-averaged readout of Section 4.4 for a finite chain."""
    n = Q.shape[0]
    B = np.zeros((2 * n, 2 * n))
    B[:n, :n] = Q
    B[:n, n:] = np.eye(n)
    out = []
    lo = 0.0
    p_lo = np.asarray(p0, dtype=np.float64)
    for b in np.asarray(edges, dtype=np.float64):
        D = b - lo
        assert D > 0.0
        E = scipy.linalg.expm(B * D)
        out.append(p_lo @ E[:n, n:] / D)
        p_lo = p_lo @ E[:n, :n]
        lo = b
    return np.stack(out)


def stationary(Q):
    """The probability row vector p with p Q = 0 (least squares with a normalisation row)."""
    n = Q.shape[0]
    A = np.vstack([Q.T, np.ones((1, n))])
    b = np.zeros(n + 1)
    b[-1] = 1.0
    p, *_ = np.linalg.lstsq(A, b, rcond=None)
    return p


def detailed_balance_chain(up, down):
    """Stationary law of a birth-death chain on 0..n: pi_{i+1}/pi_i = up[i]/down[i+1]."""
    n = len(up)
    logp = np.zeros(n)
    for i in range(n - 1):
        logp[i + 1] = logp[i] + np.log(up[i]) - np.log(down[i + 1])
    p = np.exp(logp - logp.max())
    return p / p.sum()


def immigration_death_mean(lam: float, mu: float, t):
    """Poisson mean of A(t) for 0 -> A (lam), A -> 0 (mu A) started from A = 0."""
    return lam / mu * (1.0 - np.exp(-mu * np.asarray(t, dtype=np.float64)))


def enumerate_jump_chain(net, log_rates, x0, n_jumps: int):
    """Exact law of the jump chain after n_jumps jumps.

    Returns (law, mean_time): law maps each state reachable in exactly n_jumps jumps (or an
    absorbing state reached earlier, kept in place) to its probability; mean_time[k] is the exact
    expected time of the k-th jump (E[t_k], k = 1..n_jumps, conditioned on no absorption)."""
    V = net.stoich_dense()
    frontier = {tuple(int(v) for v in x0): 1.0}
    mean_time = []
    t_acc = 0.0
    for _ in range(n_jumps):
        nxt = {}
        dt = 0.0
        for x, p in frontier.items():
            a = propensities(net, log_rates, x)
            a0 = a.sum()
            if a0 == 0:
                nxt[x] = nxt.get(x, 0.0) + p
                continue
            dt += p / a0
            for j in range(net.n_reactions):
                if a[j] > 0:
                    y = tuple(int(v) for v in np.asarray(x) + V[j])
                    nxt[y] = nxt.get(y, 0.0) + p * a[j] / a0
        t_acc += dt
        mean_time.append(t_acc)
        frontier = nxt
    return frontier, np.array(mean_time)
