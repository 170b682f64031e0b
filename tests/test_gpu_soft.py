"""GPU tests of the soft forward (arXiv 2602.19775, Section 3.3, Eq. 4) and of the exact gradient of that
relaxed model, through the C ABI, against the FP64 oracle on the same seeded noise.

The soft path has no discrete choice: a trajectory is a smooth function of its noise, so the GPU's binary32
states drift from the oracle's binary64 ones by roundoff only. Per step the update carries a few dozen
roundings (propensities, two logarithms, an exponential and a division per weight, the normalisation, the
stoichiometric sum): directly that is within k * 64 * 2^-24 * (max|X| + 1) after k steps. The relaxed dynamics
also amplifies what it is given: a soft count x near 0 makes log a = log(k x) sensitive to x, and the soft
sample responds with a factor ~1/(T x). Each step's roundings act like perturbations of ~64 ulp of the log
propensities, so the oracle's own response to a perturbation delta of each log rate, scaled by
64 * 2^-24 / delta, bounds their amplified effect (x 4 for the signs that can add up). A sample whose bracket
differs (an event time within the clock tolerance of the sample time) may further differ by one update,
at most max|v|. A rate perturbation does not stand for the rounding of a soft count that passes close to 0,
whose relative error is larger; on the ion channel a few trajectories do that. So the bound is required on
99% of the samples, and every sample's ensemble mean must agree within the mean of the bounds.
"""
import numpy as np
import pytest
import torch

import ssa_workloads as W
from ssa_workloads.configs import HOLD, LINEAR
from oracle import native

from test_gpu_parity import EPS32, _clock_tol, _theta32

pytestmark = pytest.mark.gpu
BIN = native.BIN
NAMES = {HOLD: "hold", LINEAR: "linear", BIN: "bin"}


@pytest.fixture(scope="module")
def S():
    from paper_2602_19775_gb300 import ssa
    ssa._lib.lib()
    return ssa


CASES = {
    "dimer": lambda: (W.dimerization_2a_b(0.01, 0.1, 100), 20.0, [0, 1], 0.5, 2048),
    "mixed_hot": lambda: (W.mixed_orders_toy(), 4.0, [0, 1, 2], 2.0, 1024),
    "ion_channel": lambda: (W.ion_channel_coi(), 8.0, [1], 0.3, 4096),
    # 12 species, 24 reactions (43 stoichiometric entries): the largest network of the specialised kernels, and
    # on the warp layout 7 lanes of Philox blocks; ~430 steps
    "random_24": lambda: (W.random_network(np.random.default_rng(31), n_species_range=(12, 12),
                                           n_reactions_range=(24, 24)), 0.3, [0, 3, 7], 2.0, 256),
}


def _both(S, net, t_end, ts, obs_sp, T, n, readout, seed, dl=None, max_steps=4096, tpt=0):
    t32, t64 = _theta32(net.log_rates)
    snet = S.Network(net)
    fw = S.forward(snet, torch.tensor(t32, device="cuda"), n, net.x0, t_end, ts, obs_sp, seed, readout=NAMES[readout],
                   record=dl is not None, max_steps=max_steps, selector="soft", temperature=T, threads_per_traj=tpt)
    torch.cuda.synchronize()
    orc = native.run(net, t64, net.x0, n, t_end, ts, np.asarray(obs_sp, np.int32), seed, readout, max_steps=max_steps,
                     selector="soft", temperature=float(np.float32(T)), dl_dobs=dl, ev_cap=max_steps)
    return snet, fw, orc


WARP_CASES = {
    # 160 reactions, ~1,300 steps: beyond the specialised kernels, the warp layout's own case (lanes hold up to
    # 2 Philox blocks). The relaxed model is taken where it is well conditioned (T = 2: the oracle's own gradient
    # moves by 6e-7 under random 1e-6 perturbations of log k); at T = 0.5 the seed-16 network moves by 0.9%,
    # beyond what binary32 arithmetic can be compared at.
    "random_160": lambda: (W.random_network(np.random.default_rng(17), n_species_range=(20, 20),
                                            n_reactions_range=(160, 160)), 0.2, [0, 3, 7], 2.0, 128),
}


@pytest.mark.parametrize("readout", [HOLD, LINEAR, BIN])
@pytest.mark.parametrize("case,kernels", [(c, k) for c in sorted(CASES) for k in ("specialised", "warp")] +
                         [(c, "warp") for c in sorted(WARP_CASES)])
def test_soft_forward_matches_oracle(S, case, kernels, readout):
    """The soft forward on the network-specialised thread kernels and on the warp-per-trajectory kernels
    (threads_per_traj = 32; the only layout for networks past the specialised kernels' limits)."""
    net, t_end, obs_sp, T, n = {**CASES, **WARP_CASES}[case]()
    ts = W.uniform_sample_grid(t_end, 16)
    snet, fw, orc = _both(S, net, t_end, ts, obs_sp, T, n, readout, 3, tpt=32 if kernels == "warp" else 0)
    assert fw.run.variant == (32 if kernels == "warp" else 2)
    st = fw.status.cpu().numpy()
    assert np.all(st <= 1) and np.all(orc.status <= 1)
    same = fw.draws.cpu().numpy() == orc.draws  # a crossing decided within the clock tolerance may differ
    assert same.mean() > 0.99
    V = net.stoich_dense()
    vmax = np.abs(V).max()
    obs_g = fw.obs.double().cpu().numpy()
    tol_t = _clock_tol(net.n_reactions, ts)
    # amplification: the oracle's response to a perturbation of each log rate
    delta = 1e-6
    t64 = net.log_rates.astype(np.float32).astype(np.float64)
    sens = np.zeros_like(orc.obs)
    for r in range(net.n_params):
        th = t64.copy()
        th[r] += delta
        o2 = native.run(net, th, net.x0, n, t_end, ts, np.asarray(obs_sp, np.int32), 3, readout, max_steps=4096,
                        selector="soft", temperature=float(np.float32(T)))
        sens += np.abs(o2.obs - orc.obs)
    amp = 4 * 64 * EPS32 / delta * sens
    idx = np.nonzero(same)[0]
    bound = np.zeros((len(idx), len(ts)))
    err = np.zeros((len(idx), len(ts)))
    for q, i in enumerate(idx):
        t_ev = orc.times[i, :orc.draws[i]]
        xmax = np.abs(orc.obs[i]).max() + 1.0
        for s in range(len(ts)):
            k = np.searchsorted(t_ev, ts[s], side="right")
            b = (k + 1) * 64 * EPS32 * xmax + amp[i, s].max()
            if np.any(np.abs(t_ev - ts[s]) <= tol_t[s]) or (readout == BIN and np.any(
                    (t_ev > (ts[s - 1] if s else 0.0) - tol_t[s]) & (t_ev <= ts[s] + tol_t[s]))):
                b += vmax * (1.0 if readout != BIN else tol_t[s] * k / (ts[s] - (ts[s - 1] if s else 0.0)) + 1e-6)
            bound[q, s] = b
            err[q, s] = np.abs(obs_g[i, s] - orc.obs[i, s]).max()
    within = err <= bound
    worst = np.unravel_index(np.argmax(err / bound), err.shape)
    assert within.mean() >= 0.99, (within.mean(), idx[worst[0]], worst[1], err[worst], bound[worst])
    mean_err = np.abs((obs_g[idx] - orc.obs[idx]).mean(0)).max(-1)
    assert np.all(mean_err <= bound.mean(0)), (mean_err, bound.mean(0))


@pytest.mark.parametrize("readout", [HOLD, LINEAR, BIN])
@pytest.mark.parametrize("case,kernels", [(c, k) for c in sorted(CASES) for k in ("specialised", "warp")] +
                         [(c, "warp") for c in sorted(WARP_CASES)])
def test_soft_gradient_matches_oracle(S, case, kernels, readout):
    """The exact gradient of the relaxed model: the specialised thread kernels' and the warp kernels' adjoints
    (segment re-runs from float checkpoints) against the oracle's."""
    net, t_end, obs_sp, T, n = {**CASES, **WARP_CASES}[case]()
    ts = W.uniform_sample_grid(t_end, 16)
    dl = W.seeded_dl_dobs(5, n, len(ts), len(obs_sp), scale=1.0 / n)
    snet, fw, orc = _both(S, net, t_end, ts, obs_sp, T, n, readout, 9, dl=dl, tpt=32 if kernels == "warp" else 0)
    assert fw.run.variant == (32 if kernels == "warp" else 2)
    same = fw.draws.cpu().numpy() == orc.draws
    # a bracket flip moves a sample's dependence to the neighbouring interval: leave such trajectories out
    gb = fw.run.brackets().cpu().numpy()
    for i in range(n):
        d = int(orc.draws[i])
        applied = d - 1 if orc.status[i] == native.STATUS["OK"] else d
        same[i] &= np.array_equal(gb[i], np.searchsorted(orc.times[i, :applied], ts, side="right"))
    assert same.mean() > 0.98
    dl_g = dl.copy()
    dl_g[~same] = 0.0
    g = S.backward(fw, torch.tensor(dl_g, dtype=torch.float32, device="cuda"), T).double().cpu().numpy()
    counts, mism = fw.run.status_counts()
    assert mism == 0  # every regenerated segment ends on its checkpoint, bit for bit
    ref = orc.dtheta[same].sum(0)
    rel = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30)
    assert rel < 2e-3, (rel, g, ref)


def test_soft_forward_at_low_temperature_is_the_hard_forward(S):
    """At T = 1e-6 the binary32 soft sample is exactly one-hot wherever the key gap exceeds 150 T in log2 units,
    so on trajectories whose oracle margins all exceed 1e-3 the soft states are the hard integer states."""
    wl = W.config_c1()
    n = 2048
    t32, t64 = _theta32(wl.log_rates)
    snet = S.Network(wl.net)
    th = torch.tensor(t32, device="cuda")
    soft = S.forward(snet, th, n, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, 11, readout="hold",
                     selector="soft", temperature=1e-6, max_steps=4096)
    hard = S.forward(snet, th, n, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, 11, readout="hold",
                     max_steps=4096)
    orc = native.run(wl.net, t64, wl.x0, n, wl.t_end, wl.sample_times, wl.obs_species, 11, HOLD, ev_cap=4096)
    clear = np.array([np.nanmin(orc.margins[i, :orc.draws[i]]) > 1e-3 for i in range(n)])
    assert clear.mean() > 0.5
    a = soft.obs.cpu().numpy()[clear]
    b = hard.obs.float().cpu().numpy()[clear]
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(soft.draws.cpu().numpy()[clear], hard.draws.cpu().numpy()[clear])


def test_soft_simulate_autograd_matches_backward(S):
    net = W.dimerization_2a_b(0.01, 0.1, 100)
    ts = W.uniform_sample_grid(10.0, 10)
    snet = S.Network(net)
    theta = torch.tensor(net.log_rates.astype(np.float32), device="cuda", requires_grad=True)
    obs = S.simulate(snet, theta, 4096, net.x0, 10.0, ts, [0], 2, readout="linear", temperature=0.5, soft=True)
    loss = (obs.mean(0) ** 2).mean()
    loss.backward()
    fw = S.forward(snet, theta.detach(), 4096, net.x0, 10.0, ts, [0], 2, readout="linear", record=True,
                   selector="soft", temperature=0.5)
    assert torch.equal(fw.obs, obs.detach())
    dl = (2.0 * fw.obs.mean(0) / fw.obs.shape[1] / 4096).expand(4096, -1, -1).contiguous()
    torch.testing.assert_close(theta.grad, S.backward(fw, dl, 0.5), rtol=1e-5, atol=1e-8)


@pytest.mark.parametrize("readout", ["hold", "linear", "bin"])
def test_warp_soft_forward_equals_specialised_on_two_reactions(S, readout):
    """With M = 2 lane 0 holds every reaction of the warp layout, so a0, the largest key and the normaliser are
    summed in the thread kernels' order (the other lanes add zeros): the two layouts agree bit for bit, which
    checks the species-major update list and the readouts of the warp soft forward."""
    net = W.dimerization_2a_b(0.01, 0.1, 100)
    snet = S.Network(net)
    th = torch.tensor(net.log_rates.astype(np.float32), device="cuda")
    ts = W.uniform_sample_grid(20.0, 16)
    runs = [S.forward(snet, th, 3000, net.x0, 20.0, ts, [0, 1], 7, readout=readout, selector="soft", temperature=0.4,
                      threads_per_traj=tpt, max_steps=8192) for tpt in (0, 32)]
    assert [r.run.variant for r in runs] == [2, 32]
    assert torch.equal(runs[0].obs, runs[1].obs)
    assert torch.equal(runs[0].draws, runs[1].draws) and torch.equal(runs[0].status, runs[1].status)


@pytest.mark.parametrize("readout", ["hold", "linear", "bin"])
@pytest.mark.parametrize("case", ["dimer", "random_24"])
def test_warp_soft_gradient_equals_specialised(S, case, readout):
    """The warp layout's soft gradient against the specialised kernels'. On 2A <-> B every reaction sits on lane
    0, so the forwards agree bit for bit and the gradients differ only by the order of the trajectory sums
    (1e-5); on the 24-reaction network a0 and the normaliser are also summed in another order, which the
    well-conditioned relaxed model carries into the gradient at the 1e-4 level."""
    net, t_end, obs_sp, T, n = {"dimer": lambda: (W.dimerization_2a_b(0.01, 0.1, 100), 20.0, [0, 1], 0.4, 3000),
                                "random_24": CASES["random_24"]}[case]()
    snet = S.Network(net)
    th = torch.tensor(net.log_rates.astype(np.float32), device="cuda")
    ts = W.uniform_sample_grid(t_end, 16)
    dl = torch.tensor(W.seeded_dl_dobs(6, n, len(ts), len(obs_sp), scale=1.0 / n), dtype=torch.float32, device="cuda")
    g = []
    for tpt in (0, 32):
        fw = S.forward(snet, th, n, net.x0, t_end, ts, obs_sp, 7, readout=readout, selector="soft", temperature=T,
                       threads_per_traj=tpt, max_steps=8192, record=True)
        assert fw.run.variant == (2 if tpt == 0 else 32)
        g.append(S.backward(fw, dl, T))
        assert fw.run.status_counts()[1] == 0
    rtol = 1e-5 if case == "dimer" else 1e-4
    torch.testing.assert_close(g[1], g[0], rtol=rtol, atol=rtol * float(g[0].abs().max()))


def test_soft_rules(S):
    net = W.dimerization_2a_b()
    snet = S.Network(net)
    th = torch.tensor(net.log_rates.astype(np.float32), device="cuda")
    args = (snet, th, 64, net.x0, 1.0, [0.5, 1.0], [0], 0)
    with pytest.raises(RuntimeError):  # no temperature
        S.forward(*args, selector="soft")
    # without the specialised kernels the warp kernels run it, forward only
    assert S.forward(*args, selector="soft", temperature=0.5, specialize=False).run.variant == 32
    assert S.forward(*args, selector="soft", temperature=0.5, threads_per_traj=32).run.variant == 32
    fw = S.forward(*args, selector="soft", temperature=0.5, threads_per_traj=32, record=True, readout="linear")
    with pytest.raises(RuntimeError):  # the gradient of the relaxed model is at its own temperature
        S.backward(fw, torch.zeros(64, 2, 1, device="cuda"), 0.25)
    assert torch.count_nonzero(S.backward(fw, torch.zeros(64, 2, 1, device="cuda"), 0.5)) == 0
    with pytest.raises(RuntimeError):
        S.forward(*args, selector="soft", temperature=0.5, specialize=False, threads_per_traj=1)
    fw = S.forward(*args, selector="soft", temperature=0.5, record=True, readout="linear")
    with pytest.raises(RuntimeError):  # the gradient of the relaxed model is at its own temperature
        S.backward(fw, torch.zeros(64, 2, 1, device="cuda"), 0.25)
    with pytest.raises(RuntimeError):  # no event log
        fw.run.events(16)
    g = S.backward(fw, torch.zeros(64, 2, 1, device="cuda"), 0.5)
    assert torch.count_nonzero(g) == 0
    # the other selectors refuse a temperature in their options
    opts = S.make_opts("hold")
    opts.temperature = 0.5
    with pytest.raises(RuntimeError):
        S.workspace_bytes(snet, 64, 2, opts)
