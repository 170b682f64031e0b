"""Parameter inference through the library. Section 4.1 (and 4.4): fit the log rate constants of a network
so that the ensemble-mean observables of simulated trajectories match a target, with the
straight-through gradient of the exact SSA, RMSprop on theta = log k, and the temperature and the learning
rate annealed geometrically over the iterations (Section 4.1 anneals T from 1.0 to 0.001 with a geometric
learning-rate decay). The estimator's variance grows as T falls: on the 2A <-> B workload (about 250 draws
per trajectory) single-batch gradients at T = 0.01 reach 1e7 where T = 0.1 gives ~2e2, so the learning rate
has to fall with T.

Section 4.2, the start-point map: states sampled along one long reference trajectory start short
replicated segments, whose rates of change of the observed species are matched to the targets while only
some rates are trained (reference_start_points, segment_rates, fit_start_point_map). On the oscillator with
five protein rates trained, the paper's RMSprop diverges here: its per-parameter normalisation moves every
rate at the same speed, but the production and degradation of A are strongly coupled (at rates 20-30% off,
the gradient pushes the degradation rate further off until the production rate is close), and the complex
formation rate gammaC is weakly determined, its straight-through gradient biased (at T = 0.1, about 20x its
finite-difference value). Plain gradient descent follows the large gradient components first; with its
largest per-parameter step clipped (optimizer "sgd") it recovers all five rates.

The simulation and its gradient run in the library (simulate / SSAFunction); this module is the host-side
loop around them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from .ssa import Network, forward, simulate


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


def reference_start_points(net: Network, theta, x0, n_points: int, t_ref: float, seed: int,
                           max_steps: int = 1 << 24) -> np.ndarray:
    """Start points of the start-point map (Section 4.2): the states of one long reference trajectory
    (simulated at theta) at n_points uniformly random times in (0, t_ref], in time order; int32 [n_points, N]."""
    rng = np.random.default_rng(seed)
    times = np.sort(rng.uniform(0.0, t_ref, n_points))
    theta = torch.as_tensor(np.asarray(theta, dtype=np.float32), device="cuda")
    fw = forward(net, theta, 1, x0, t_ref, times, list(range(net.n_species)), seed, readout="hold",
                 max_steps=max_steps)
    if int(fw.status[0]) > 1:
        raise RuntimeError(f"reference trajectory stopped with status {int(fw.status[0])}")
    return fw.obs[0].cpu().numpy().astype(np.int32)


def segment_rates(net: Network, theta: torch.Tensor, starts, replicates: int, horizon: float, obs_species, seed: int,
                  temperature: float, max_steps: int = 4096) -> torch.Tensor:
    """Rates of change of the start-point map (Section 4.2), differentiable in theta: from each start point,
    `replicates` segments of length `horizon`; the rate of observable c is (the ensemble mean of its exact
    average over the final two thirds of the segment - its start value) / (2 horizon / 3), the time from the
    start to the middle of that window. Returns [n_points, n_obs]."""
    starts = torch.as_tensor(np.asarray(starts, dtype=np.int32), device="cuda")
    x0 = starts.repeat_interleave(replicates, dim=0)
    edges = [horizon / 3.0, horizon]
    obs = simulate(net, theta, x0.shape[0], x0, horizon, edges, obs_species, seed, readout="bin",
                   temperature=temperature, max_steps=max_steps)
    window = obs[:, 1, :].reshape(starts.shape[0], replicates, -1).mean(1)
    start = starts[:, torch.as_tensor(np.asarray(obs_species), device="cuda").long()].float()
    return (window - start) / (2.0 * horizon / 3.0)


def fit_start_point_map(net: Network, theta0, trainable, starts, target_rates, obs_species, horizon: float,
                        replicates: int, batch: int, iters: int, temperature: float, lr: float = 0.1,
                        lr_final: float | None = None, seed0: int = 0, optimizer: str = "rmsprop",
                        max_step: float | None = 0.05) -> tuple[np.ndarray, FitHistory]:
    """Gradient steps on the trainable log rates (the others stay at theta0) to match the segment rates of a
    batch of start points per iteration to their targets (mean squared error), at a fixed temperature with a
    geometric learning-rate decay (Section 4.2). target_rates: [n_points, n_obs] for the rows of `starts`.
    optimizer: "rmsprop" (the paper's), "adam", or "sgd": theta -= lr * gradient, scaled down where needed so
    that no parameter moves by more than max_step (log units; None: no clip)."""
    if optimizer not in ("rmsprop", "adam", "sgd"):
        raise ValueError("optimizer must be rmsprop, adam or sgd")
    dev = torch.device("cuda")
    base = torch.tensor(np.asarray(theta0, dtype=np.float32), device=dev)
    mask = torch.zeros_like(base)
    mask[list(trainable)] = 1.0
    free = torch.zeros_like(base, requires_grad=True)
    opt = (torch.optim.RMSprop([free], lr=lr) if optimizer == "rmsprop" else
           torch.optim.Adam([free], lr=lr) if optimizer == "adam" else None)
    tgt = torch.as_tensor(np.asarray(target_rates, dtype=np.float32), device=dev)
    starts = np.asarray(starts)
    rng = np.random.default_rng(seed0)
    lr_final = lr if lr_final is None else lr_final
    hist = FitHistory()
    for it in range(iters):
        frac = it / max(iters - 1, 1)
        cur_lr = lr * (lr_final / lr) ** frac
        if opt is not None:
            for grp in opt.param_groups:
                grp["lr"] = cur_lr
        rows = rng.choice(starts.shape[0], size=batch, replace=False)
        theta = base + mask * free
        rates = segment_rates(net, theta, starts[rows], replicates, horizon, obs_species, seed0 + 1 + it, temperature)
        loss = ((rates - tgt[torch.as_tensor(rows, device=dev)]) ** 2).mean()
        free.grad = None
        loss.backward()
        if opt is not None:
            opt.step()
        else:
            with torch.no_grad():
                step = cur_lr * free.grad
                big = float(step.abs().max())
                if max_step is not None and big > max_step:
                    step *= max_step / big
                free -= step
        hist.loss.append(float(loss.item()))
        hist.theta.append((base + mask * free).detach().double().cpu().numpy())
        hist.temperature.append(temperature)
    return (base + mask * free).detach().double().cpu().numpy(), hist
