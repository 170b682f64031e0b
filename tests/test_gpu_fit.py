"""End-to-end inference on a synthetic target (Section 4.1's dimerization recovery on the 2A <-> B
workload): RMSprop on log k through the straight-through gradient, temperature annealed 1.0 -> 0.05 and the
learning rate 0.05 -> 0.005, recovers the rates that generated the target from a start off by a factor of two
in each."""
import numpy as np
import pytest
import torch

import ssa_workloads as W

pytestmark = pytest.mark.gpu


def test_dimerization_rates_are_recovered():
    from paper_2602_19775_gb300 import ssa
    from paper_2602_19775_gb300.fit import fit_ensemble_mean
    wl = W.config_c2()
    net = ssa.Network(wl.net)
    true = np.log([0.01, 0.1])
    tfw = ssa.forward(net, torch.tensor(true.astype(np.float32), device="cuda"), 65536, wl.x0, wl.t_end,
                      wl.sample_times, wl.obs_species, 1, readout="linear", max_steps=4096)
    target = ssa.ensemble_mean(tfw.obs).cpu().numpy()
    theta, hist = fit_ensemble_mean(net, wl.log_rates, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, target,
                                    n_traj=8192, iters=60, lr=0.05, lr_final=0.005, t_start=1.0, t_final=0.05,
                                    max_steps=4096)
    assert hist.loss[-1] < 0.01 * hist.loss[0], (hist.loss[0], hist.loss[-1])
    assert np.all(np.abs(theta - true) < 0.05), (theta, true)
