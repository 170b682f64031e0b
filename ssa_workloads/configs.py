"""Workload configurations (seeded, synthetic).

* C1  2A <-> B, k = (0.01, 0.1), A0 = 100, 1,024 trajectories, t_end = 50, 50 samples, seed 0,
      HOLD readout of A and B; forward only.
* C2  the same network with the straight-through gradient: 65,536 trajectories, LINEAR readout
      of A, evaluated at k = (0.02, 0.05), checkpoint interval K = 64, T in {0.1, 0.5, 1.0};
      loss = mean over samples of (ensemble mean A(t_s) - target_s)^2.
* C3  the activator-repressor oscillator, 2^20 trajectories to t_end = 400 with 400 samples of R.

Sample grids are t_s = s * t_end / S for s = 1..S (t_end included, 0 excluded).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .networks import NetworkSpec, dimerization_2a_b, vilar_oscillator, random_network

HOLD = 0
LINEAR = 1


def uniform_sample_grid(t_end: float, S: int) -> np.ndarray:
    """t_end/S, 2 t_end/S, ..., t_end; S * (t_end / S) can round one ulp above t_end, so clip."""
    return np.minimum(np.arange(1, S + 1, dtype=np.float64) * (t_end / S), float(t_end))


@dataclass
class Workload:
    name: str
    net: NetworkSpec
    log_rates: np.ndarray       # float64 [P]
    x0: np.ndarray              # int32 [N]
    n_traj: int
    t_end: float
    sample_times: np.ndarray    # float64 [S]
    obs_species: np.ndarray     # int32 [n_obs]
    seed: int
    readout: int
    ckpt_interval: int = 64
    temperatures: tuple = ()
    max_steps: int = 1 << 20


def config_c1(n_traj: int = 1024) -> Workload:
    net = dimerization_2a_b(0.01, 0.1, 100)
    return Workload("c1_dimer_2a_b_fwd", net, net.log_rates.copy(), net.x0.copy(), n_traj, 50.0,
                    uniform_sample_grid(50.0, 50), np.array([0, 1], np.int32), 0, HOLD,
                    max_steps=4096)


def config_c2(n_traj: int = 65536) -> Workload:
    net = dimerization_2a_b(0.01, 0.1, 100)
    theta = np.log(np.array([0.02, 0.05], dtype=np.float64))
    return Workload("c2_dimer_2a_b_fwd_adj", net, theta, net.x0.copy(), n_traj, 50.0,
                    uniform_sample_grid(50.0, 50), np.array([0], np.int32), 0, LINEAR,
                    ckpt_interval=64, temperatures=(0.1, 0.5, 1.0), max_steps=4096)


def config_c3(n_traj: int = 1 << 20, t_end: float = 400.0, S: int = 400) -> Workload:
    net = vilar_oscillator()
    return Workload("c3_vilar_oscillator", net, net.log_rates.copy(), net.x0.copy(), n_traj, t_end,
                    uniform_sample_grid(t_end, S), np.array([net.species_index("R")], np.int32), 0,
                    LINEAR, ckpt_interval=64, temperatures=(0.1,), max_steps=1 << 22)


def seeded_dl_dobs(seed: int, n_traj: int, S: int, n_obs: int, scale: float = 1.0) -> np.ndarray:
    """Seeded upstream gradient dL/dobs [n_traj, S, n_obs] (float64) for parity cases."""
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal((n_traj, S, n_obs))).astype(np.float64)


@dataclass
class BatchWorkload:
    name: str
    nets: list                  # NetworkSpec per network
    n_traj: np.ndarray          # int64 [n_nets]
    t_end: float
    sample_times: np.ndarray    # float64 [S], shared by every network
    obs_species: list           # int32 arrays, per network
    loss_weights: list          # float64 [S, n_obs] per network: L = sum c * mean over trajectories of obs
    seed: int
    readout: int
    temperature: float
    draw_index: np.ndarray      # int64 [n_nets]: position of each accepted network in the generator stream


def config_c4(n_nets: int = 256, traj_scale: float = 1.0, rejected=(), seed: int = 3, n_obs_max: int = 8
              ) -> BatchWorkload:
    """Uneven batch of random mass-action networks (one seeded stream, `seed`): N ~ U{2..64},
    M ~ U{4..512} (random_network), trajectories per network log-uniform in [256, 65,536] scaled by
    traj_scale (at least 1), t_end = 10, 20 uniform samples, LINEAR readout, T = 0.5. Networks are drawn
    one after another from the stream; a draw whose position is in `rejected` (the redraw list of an
    oracle pilot) is skipped and the next draw takes its place. Observed species: the first
    min(N, n_obs_max). Loss weights c ~ N(0, 1) (seed 4)."""
    rng = np.random.default_rng(seed)
    trng = np.random.default_rng(seed + 1000)
    crng = np.random.default_rng(4)
    rejected = set(int(r) for r in rejected)
    nets, idx = [], []
    d = 0
    while len(nets) < n_nets:
        net = random_network(rng, n_species_range=(2, 64), n_reactions_range=(4, 512))
        if d not in rejected:
            nets.append(net)
            idx.append(d)
        d += 1
    n = np.exp(trng.uniform(np.log(256.0), np.log(65536.0), size=n_nets))
    n_traj = np.maximum(1, np.round(n * traj_scale)).astype(np.int64)
    ts = uniform_sample_grid(10.0, 20)
    obs = [np.arange(min(net.n_species, n_obs_max), dtype=np.int32) for net in nets]
    c = [crng.standard_normal((len(ts), len(o))) for o in obs]
    return BatchWorkload("c4_uneven_batch", nets, n_traj, 10.0, ts, obs, c, seed, LINEAR, 0.5,
                         np.array(idx, np.int64))
