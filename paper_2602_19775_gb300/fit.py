"""Parameter inference through the library (arXiv 2602.19775, Section 4.1): fit the log rate constants
of a network so that the ensemble-mean observables of simulated trajectories match a target, with the
straight-through gradient of the exact SSA, RMSprop on theta = log k, and the temperature and the learning
rate annealed geometrically over the iterations (Section 4.1 anneals T from 1.0 to 0.001 with a geometric
learning-rate decay). The estimator's variance grows as T falls: on the 2A <-> B workload (about 250 draws
per trajectory) single-batch gradients at T = 0.01 reach 1e7 where T = 0.1 gives ~2e2, so the learning rate
has to fall with T.

The simulation and its gradient run in the library (simulate / SSAFunction); this module is the host-side
loop around them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from .ssa import Network, simulate


@dataclass
class FitHistory:
    loss: list = field(default_factory=list)
    theta: list = field(default_factory=list)
    temperature: list = field(default_factory=list)


def fit_ensemble_mean(net: Network, theta0, x0, t_end: float, sample_times, obs_species, target, n_traj: int,
                      iters: int, lr: float = 0.05, lr_final: float | None = None, t_start: float = 1.0,
                      t_final: float = 0.001, seed0: int = 0, readout: str = "linear",
                      max_steps: int = 1 << 14) -> tuple[np.ndarray, FitHistory]:
    """Minimise mean_s,o (ensemble mean obs - target)^2 over theta = log k.

    target: [S, n_obs] (array or tensor). Each iteration simulates n_traj fresh trajectories (seed
    seed0 + iteration). The temperature goes geometrically from t_start to t_final and the learning rate
    from lr to lr_final (default: constant). Returns the final theta (float64 numpy) and the history of
    loss, theta and T.
    """
    dev = torch.device("cuda")
    theta = torch.tensor(np.asarray(theta0, dtype=np.float32), device=dev, requires_grad=True)
    tgt = torch.as_tensor(np.asarray(target, dtype=np.float32), device=dev)
    opt = torch.optim.RMSprop([theta], lr=lr)
    hist = FitHistory()
    lr_final = lr if lr_final is None else lr_final
    for it in range(iters):
        frac = it / max(iters - 1, 1)
        T = t_start * (t_final / t_start) ** frac
        for grp in opt.param_groups:
            grp["lr"] = lr * (lr_final / lr) ** frac
        obs = simulate(net, theta, n_traj, x0, t_end, sample_times, obs_species, seed0 + it, readout=readout,
                       temperature=T, max_steps=max_steps)
        loss = ((obs.mean(0) - tgt) ** 2).mean()
        opt.zero_grad()
        loss.backward()
        opt.step()
        hist.loss.append(float(loss.item()))
        hist.theta.append(theta.detach().double().cpu().numpy())
        hist.temperature.append(T)
    return theta.detach().double().cpu().numpy(), hist
