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

from .networks import NetworkSpec, dimerization_2a_b, vilar_oscillator

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
