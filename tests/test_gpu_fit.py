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


def test_ion_channel_rates_from_bin_averages():
    """Section 4.4 on a synthetic target: the mean open count of two C <-> O -> I channels, averaged
    exactly over 800 bins of 0.01 ms, generated at k = (0.75, 0.1, 1.2) per ms. From (0.3, 0.4, 0.5) the
    opening and inactivation rates are recovered; the closing rate is weakly identified by the mean
    alone (the paper also sees it converge last) and only has to move towards its true value."""
    from paper_2602_19775_gb300 import ssa
    from paper_2602_19775_gb300.fit import fit_ensemble_mean
    spec = W.ion_channel_coi()
    net = ssa.Network(spec)
    ts = W.uniform_sample_grid(8.0, 800)
    true = spec.log_rates.astype(np.float32).astype(np.float64)
    target = ssa.forward(net, torch.tensor(true, dtype=torch.float32, device="cuda"), 1 << 20, spec.x0, 8.0, ts,
                         [1], 12345, readout="bin", max_steps=64).obs.mean(0).cpu().numpy()
    theta0 = np.log([0.3, 0.4, 0.5])
    theta, hist = fit_ensemble_mean(net, theta0, spec.x0, 8.0, ts, [1], target, n_traj=262144, iters=150, lr=0.05,
                                    lr_final=0.005, t_start=0.5, t_final=0.05, readout="bin", max_steps=64, seed0=7)
    assert hist.loss[-1] < 0.01 * hist.loss[0], (hist.loss[0], hist.loss[-1])
    assert abs(theta[0] - true[0]) < 0.1 and abs(theta[2] - true[2]) < 0.05, (np.exp(theta), np.exp(true))
    assert np.exp(theta[1]) < 0.38, np.exp(theta)


def test_start_point_map_segments():
    """Section 4.2's start-point map on the oscillator, as built here: start points from one reference
    trajectory, replicated segments of horizon 0.05 (about 150 draws), rates of A, R and C from the exact
    average over the final two thirds of each segment. At the true rates the segment rates agree with
    independently simulated targets (mean over start points within 4 SE per species); the map separates the
    true rates from the five protein rates perturbed by 20-30%; the straight-through gradient of the loss is
    finite at T = 3e-6."""
    from paper_2602_19775_gb300 import ssa
    from paper_2602_19775_gb300.fit import reference_start_points, segment_rates
    spec = W.vilar_oscillator()
    net = ssa.Network(spec)
    true = spec.log_rates.astype(np.float32).astype(np.float64)
    names = list(spec.param_names)
    train = [names.index(x) for x in ("betaA", "betaR", "deltaA", "deltaR", "gammaC")]
    starts = reference_start_points(net, true, spec.x0, 4096, 400.0, 1)
    assert starts.shape == (4096, 9) and np.all(starts >= 0)
    obs, H = [6, 7, 8], 0.05
    th_true = torch.tensor(true, dtype=torch.float32, device="cuda")
    with torch.no_grad():
        tgt = torch.cat([segment_rates(net, th_true, starts[i:i + 1024], 256, H, obs, 999 + i, 0.1)
                         for i in range(0, 4096, 1024)])
        sim = segment_rates(net, th_true, starts, 32, H, obs, 7, 0.1)
    d = (sim - tgt).double().cpu().numpy()
    z = d.mean(0) / (d.std(0, ddof=1) / np.sqrt(d.shape[0]))
    assert np.all(np.abs(z) < 4.0), z
    theta0 = true.copy()
    theta0[train] += np.log([1.3, 0.75, 1.25, 0.8, 1.3])
    th0 = torch.tensor(theta0, dtype=torch.float32, device="cuda", requires_grad=True)
    r0 = segment_rates(net, th0, starts, 32, H, obs, 7, 3e-6)
    loss0 = ((r0 - tgt) ** 2).mean()
    loss_true = float(((sim - tgt) ** 2).mean())
    assert float(loss0) > 3.0 * loss_true, (float(loss0), loss_true)
    loss0.backward()
    assert torch.all(torch.isfinite(th0.grad)) and float(th0.grad[train].abs().sum()) > 0


def test_start_point_map_fit_recovers_the_protein_rates():
    """Section 4.2's start-point map fit on the oscillator: the five protein rates perturbed by 20-30% and
    trained together from 2,048 start points (256 per step, 16 replicates each) at T = 0.1, by gradient
    descent with the largest per-parameter step clipped to 0.05 log units. The paper's RMSprop diverges on
    this objective (every rate moves at the same speed although the production and degradation of A are
    strongly coupled and gammaC's gradient is small and biased); gradient descent follows the large
    components first. On the CPU oracle this recipe ended, over three seeds, within 5% of the true rates
    (gammaC within 8%) after 300 steps; required here: within 10% (gammaC within 20%) and the loss at least
    halved."""
    from paper_2602_19775_gb300 import ssa
    from paper_2602_19775_gb300.fit import fit_start_point_map, reference_start_points, segment_rates
    spec = W.vilar_oscillator()
    net = ssa.Network(spec)
    true = spec.log_rates.astype(np.float32).astype(np.float64)
    names = list(spec.param_names)
    train = [names.index(x) for x in ("betaA", "betaR", "deltaA", "deltaR", "gammaC")]
    starts = reference_start_points(net, true, spec.x0, 2048, 400.0, 1)
    obs, H = [6, 7, 8], 0.05
    th_true = torch.tensor(true, dtype=torch.float32, device="cuda")
    with torch.no_grad():
        tgt = torch.cat([segment_rates(net, th_true, starts[i:i + 512], 128, H, obs, 999 + i, 0.1)
                         for i in range(0, 2048, 512)])
    theta0 = true.copy()
    theta0[train] += np.log([1.3, 0.75, 1.25, 0.8, 1.3])
    theta, hist = fit_start_point_map(net, theta0, train, starts, tgt.cpu().numpy(), obs, H, replicates=16,
                                      batch=256, iters=300, temperature=0.1, lr=2e-6, seed0=5, optimizer="sgd",
                                      max_step=0.05)
    ratio = np.exp(theta[train] - true[train])
    assert np.all(np.abs(ratio[:4] - 1.0) < 0.1) and abs(ratio[4] - 1.0) < 0.2, ratio
    assert np.mean(hist.loss[-50:]) < 0.5 * hist.loss[0], (hist.loss[0], np.mean(hist.loss[-50:]))
