"""The literal straight-through graph of Eq. 5 in float64 PyTorch CPU autograd.  Test infrastructure.

For one trajectory whose event sequence is given (the hard choices j_k of the forward), this
module rebuilds the surrogate computational graph of arXiv 2602.19775 exactly as Section 3.5
describes it: propensities a(X_k; theta) from a real-valued state, the Gumbel perturbations of
the same noise, the soft sample of Eq. 3, y_ST = y~ + stopgrad(onehot(j_k) - y~) (Eq. 5),
X_{k+1} = X_k + y_ST V (whose value is Eq. 6 and whose derivative is Eq. 7), the reparametrised
waiting time tau_k = -ln(u_0)/a0 (Section 3.1), t_{k+1} = t_k + tau_k, and the HOLD or LINEAR
readout (Section 4.1) or the exact bin average (Section 4.4: the cumulative integral of the step
path at the bin edges, differenced and divided by the bin width, with the event times as graph
nodes). Autograd then gives dL/dtheta for L = sum(c * obs), with no hand-written
derivative anywhere. Reactions with a_j = 0 are masked from the softmax (y~_j = 0) with a
gradient-safe double `where`; they still enter a0.

It is slow (one small tensor op per step) and only meant for trajectories of a few hundred steps.
"""
from __future__ import annotations

import numpy as np
import torch

from .native import BIN, HOLD, LINEAR, uniforms


def _h(reactants, X):
    r = [int(s) for s in reactants if s >= 0]
    if len(r) == 0:
        return torch.ones((), dtype=torch.float64)
    if len(r) == 1:
        return X[r[0]]
    if r[0] == r[1]:
        return X[r[0]] * (X[r[0]] - 1.0) / 2.0
    return X[r[0]] * X[r[1]]


def st_gradient(net, log_rates, x0, events, n_states: int, crossed: bool, seed: int, traj: int,
                t_end: float, sample_times, obs_species, readout: int, dl_dobs, temperature: float,
                soft: bool = False):
    """dL/dtheta of L = sum(dl_dobs * obs) through the literal Eq.-5 graph of one trajectory.

    events: the hard choices j_0..j_{n_draws-1}; n_states: number of visited states; crossed:
    whether the last draw crossed t_end (made but not applied). soft: the relaxed forward of Eq. 4
    instead (the update is the soft sample itself, real-valued states, negative mass-action factors
    clipped to 0)."""
    theta = torch.tensor(np.asarray(log_rates, dtype=np.float64), requires_grad=True)
    k_rates = torch.exp(theta)[torch.as_tensor(net.rate_index, dtype=torch.long)]
    V = torch.as_tensor(net.stoich_dense(), dtype=torch.float64)
    M = net.n_reactions
    X = torch.as_tensor(np.asarray(x0, dtype=np.float64))
    t = torch.zeros((), dtype=torch.float64)
    states, times, taus, nexts = [X], [t], [], []
    n_draws = len(events)
    for k in range(n_draws):
        u = torch.as_tensor(uniforms(seed, traj, k, M + 1))
        hs = [_h(net.reactants[j], X) for j in range(M)]
        if soft:
            hs = [torch.clamp(h, min=0.0) for h in hs]
        a = torch.stack([k_rates[j] * hs[j] for j in range(M)])
        a0 = a.sum()
        tau = -torch.log(u[0]) / a0
        active = a > 0
        safe_a = torch.where(active, a, torch.ones_like(a))
        G = -torch.log(-torch.log(u[1:]))
        z = torch.where(active, (torch.log(safe_a) + G) / temperature,
                        torch.full_like(a, -float("inf")))
        y_soft = torch.softmax(z, dim=0)
        y_hard = torch.zeros(M, dtype=torch.float64)
        y_hard[int(events[k])] = 1.0
        y_st = y_soft if soft else y_soft + (y_hard - y_soft).detach()   # Eq. 4 or Eq. 5
        X_next = X + y_st @ V                              # Eqs. 6 and 7
        t_next = t + tau
        taus.append(tau)
        nexts.append(X_next)
        if k + 1 < n_states:                               # applied draw
            X, t = X_next, t_next
            states.append(X)
            times.append(t)
    assert len(states) == n_states
    obs = []
    tvals = [float(tt) for tt in times]
    sel = torch.as_tensor(np.asarray(obs_species), dtype=torch.long)

    def bracket(b):
        k = 0
        while k + 1 < n_states and tvals[k + 1] <= b:
            k += 1
        return k

    def cumulative(b):
        # int_0^b X(t) dt of the right-continuous step path, through the graph's times
        k = bracket(b)
        c = states[k] * (b - times[k])
        for q in range(k):
            c = c + states[q] * (times[q + 1] - times[q])
        return c

    if readout == BIN:
        lo = 0.0
        for b in np.asarray(sample_times, dtype=np.float64):
            obs.append(((cumulative(float(b)) - cumulative(lo)) / (float(b) - lo))[sel])
            lo = float(b)
    for ts in (np.asarray(sample_times, dtype=np.float64) if readout != BIN else ()):
        k = 0
        while k + 1 < n_states and tvals[k + 1] <= ts:
            k += 1
        has_next = k < n_draws and (k + 1 < n_states or crossed)
        Xk = states[k]
        if readout == LINEAR and has_next:
            alpha = (float(ts) - times[k]) / taus[k]
            val = Xk + alpha * (nexts[k] - Xk)
        else:
            val = Xk
        obs.append(val[sel])
    obs = torch.stack(obs) if obs else torch.zeros((0, len(obs_species)), dtype=torch.float64)
    L = (torch.as_tensor(np.asarray(dl_dobs, dtype=np.float64)) * obs).sum()
    if not L.requires_grad:  # a path that never moves: the readout does not depend on theta
        return np.zeros_like(theta.detach().numpy()), obs.detach().numpy()
    L.backward()
    return theta.grad.detach().numpy().copy(), obs.detach().numpy()


def grn_st_gradient(params, x, events, n_states: int, crossed: bool, seed: int, traj: int, sample_times,
                    dl_dobs, temperature: float, soft: bool = False):
    """dL/d(W1, b1, W2, b2, log_d) of L = sum(dl_dobs * obs) through the literal straight-through
    graph of one GRN trajectory (HOLD readout of the outputs), by float64 autograd. soft: the relaxed graph
    of Eq. 4 (the update is the soft sample itself; a negative count degrades at rate 0)."""
    W1 = torch.tensor(np.asarray(params.W1, np.float64), requires_grad=True)
    b1 = torch.tensor(np.asarray(params.b1, np.float64), requires_grad=True)
    W2 = torch.tensor(np.asarray(params.W2, np.float64), requires_grad=True)
    b2 = torch.tensor(np.asarray(params.b2, np.float64), requires_grad=True)
    ld = torch.tensor(np.asarray(params.log_d, np.float64), requires_grad=True)
    nh, no = W1.shape[0], W2.shape[0]
    nd = nh + no
    M = 2 * nd
    xin = torch.as_tensor(np.asarray(x, np.float64))
    E1 = W1 @ xin + b1
    V = torch.zeros((M, nd), dtype=torch.float64)
    for s in range(nd):
        V[s, s] = 1.0
        V[nd + s, s] = -1.0
    X = torch.zeros(nd, dtype=torch.float64)
    t = 0.0
    states, times = [X], [0.0]
    for k in range(len(events)):
        u = torch.as_tensor(uniforms(seed, traj, k, M + 1))
        E2 = W2 @ X[:nh] + b2
        Xd = torch.clamp(X, min=0.0) if soft else X
        a = torch.cat([params.k_max * torch.sigmoid(E1), params.k_max * torch.sigmoid(E2), torch.exp(ld) * Xd])
        a0 = a.sum()
        tau = -torch.log(u[0]) / a0
        active = a > 0
        safe_a = torch.where(active, a, torch.ones_like(a))
        G = -torch.log(-torch.log(u[1:]))
        z = torch.where(active, (torch.log(safe_a) + G) / temperature, torch.full_like(a, -float("inf")))
        y_soft = torch.softmax(z, dim=0)
        y_hard = torch.zeros(M, dtype=torch.float64)
        y_hard[int(events[k])] = 1.0
        y_st = y_soft if soft else y_soft + (y_hard - y_soft).detach()
        X_next = X + y_st @ V
        t_next = t + float(tau)
        if k + 1 < n_states:
            X, t = X_next, t_next
            states.append(X)
            times.append(t)
    obs = []
    for ts in np.asarray(sample_times, dtype=np.float64):
        k = 0
        while k + 1 < n_states and times[k + 1] <= ts:
            k += 1
        obs.append(states[k][nh:])
    obs = torch.stack(obs)
    L = (torch.as_tensor(np.asarray(dl_dobs, np.float64)) * obs).sum()
    L.backward()
    return {"W1": W1.grad.numpy().copy(), "b1": b1.grad.numpy().copy(), "W2": W2.grad.numpy().copy(),
            "b2": b2.grad.numpy().copy(), "log_d": ld.grad.numpy().copy()}
