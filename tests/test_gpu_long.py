"""Long trajectories on the GPU against the FP64 oracle.

The activator-repressor oscillator of Section 4.2 at its configured horizon: t_end = 400 with 400
LINEAR samples of R, about 1.1e6 draws per trajectory. Over that many draws the straight-through
recursion (Figure 1) grows dL/dX geometrically: the oracle's binary64 gradient of one trajectory reaches
1e40-1e75 at T = 0.1, beyond the binary32 range. `ssa_backward_wide` carries a power-of-two exponent per
trajectory and sums in binary64; it must match the oracle to 1e-3 (norm) on the trajectories whose events
agree, with the upstream gradient of the samples whose bracket flips (an event within the binary32 clock
drift of the sample time) zeroed on both sides. Event sequences follow the long-trajectory rule: every first divergence at a
near-tie of the race, and no more divergent trajectories than the oracle has steps with margin < 1e-6.
"""
import numpy as np
import pytest
import torch

import ssa_workloads as W
from oracle import native
from test_gpu_parity import GRAD_RTOL, _bracket_flips, _compare_events, _oracle_theta

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2602_19775_gb300 import ssa
    ssa._lib.lib()
    return ssa


def test_oscillator_full_horizon_gradient_matches_oracle(S):
    wl = W.config_c3(n_traj=32)
    n, T, cap, seed = wl.n_traj, 0.1, 1_500_000, 17
    t32 = wl.log_rates.astype(np.float32)
    ts = wl.sample_times
    net = S.Network(wl.net)
    fw = S.forward(net, torch.tensor(t32, device="cuda"), n, wl.x0, wl.t_end, ts, wl.obs_species, seed,
                   readout="linear", record=True, max_steps=cap, ckpt_interval=64)
    torch.cuda.synchronize()
    assert fw.run.variant == 2
    orc = native.run(wl.net, _oracle_theta(t32), wl.x0, n, wl.t_end, ts, wl.obs_species, seed, native.LINEAR,
                     max_steps=cap, ev_cap=cap)
    assert np.all(orc.status == 0) and np.all(fw.status.cpu().numpy() == 0)
    assert orc.draws.min() > 9e5
    same = _compare_events(orc, fw, fw.run.events(cap).cpu().numpy(), wl.t_end, wl.net.n_reactions, floor=None)
    assert same.sum() >= n // 2, same.sum()
    flip = _bracket_flips(orc, fw, ts, wl.net.n_reactions)
    assert flip[same].mean() < 0.25, flip[same].mean()
    # the upstream gradient of the trajectories whose events agree, without their flipped samples
    keep = same[:, None] & ~flip
    dl = W.seeded_dl_dobs(13, n, len(ts), 1, scale=1.0 / n) * keep[:, :, None]
    orc_g = native.run(wl.net, _oracle_theta(t32), wl.x0, n, wl.t_end, ts, wl.obs_species, seed, native.LINEAR,
                       max_steps=cap, dl_dobs=dl, temperature=T)
    ref = orc_g.dtheta.sum(0)
    assert np.all(np.isfinite(ref))
    assert np.abs(ref).max() > 3.4e38  # beyond binary32: the case the exponent carries
    g = S.backward_wide(fw, torch.tensor(dl, dtype=torch.float32, device="cuda"), T).cpu().numpy()
    _, mism = fw.run.status_counts()
    assert mism == 0
    assert np.all(np.isfinite(g))
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel < GRAD_RTOL, (rel, g, ref)
    big = np.abs(ref) > 1e-3 * np.linalg.norm(ref)
    np.testing.assert_allclose(g[big], ref[big], rtol=2 * GRAD_RTOL)


@pytest.mark.parametrize("readout", ["hold", "linear"])
def test_wide_adjoint_equals_plain_adjoint_in_range(S, readout):
    """Where the binary32 walk stays in range (2A <-> B, ~400 draws) the exponent stays 0 and the wide
    adjoint is the plain one summed in binary64: equal to binary32 rounding of the sum."""
    wl = W.config_c2(n_traj=3000)
    net = S.Network(wl.net)
    fw = S.forward(net, torch.tensor(wl.log_rates.astype(np.float32), device="cuda"), wl.n_traj, wl.x0, wl.t_end,
                   wl.sample_times, wl.obs_species, 4, readout=readout, record=True, max_steps=4096)
    dl = torch.tensor(W.seeded_dl_dobs(3, wl.n_traj, len(wl.sample_times), 1, scale=1.0 / wl.n_traj),
                      dtype=torch.float32, device="cuda")
    for T in (0.1, 1.0):
        a = S.backward(fw, dl, T).double().cpu().numpy()
        b = S.backward_wide(fw, dl, T).cpu().numpy()
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max(), (T, a, b)
    # a shared upstream gradient (stride 0) as well
    a = S.backward(fw, dl[0], 0.5).double().cpu().numpy()
    b = S.backward_wide(fw, dl[0], 0.5).cpu().numpy()
    assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()


def test_wide_adjoint_refuses_other_runs(S):
    from paper_2602_19775_gb300 import SSAError
    spec = W.dimerization_2a_b()
    net = S.Network(spec)
    theta = torch.tensor(spec.log_rates.astype(np.float32), device="cuda")
    fw = S.forward(net, theta, 64, spec.x0, 5.0, [1.0, 5.0], [0], 1, readout="linear", record=True,
                   max_steps=4096, specialize=False)
    with pytest.raises(SSAError):
        S.backward_wide(fw, torch.zeros((64, 2, 1), device="cuda"), 0.5)


@pytest.mark.parametrize("case,readout", [("dimer", "linear"), ("mixed_orders", "hold"), ("oscillator", "linear")])
def test_multi_temperature_walk_equals_one_walk_per_temperature(S, case, readout):
    """One walk for several temperatures gives, row by row, the single-temperature gradients to binary32
    rounding (the two kernels may contract products into fused multiply-adds differently): fused for 2 and 3
    temperatures, 3 + 1 for 4, and one walk each on the generic kernels (there bit for bit)."""
    spec, t_end, n = {"dimer": (W.dimerization_2a_b(), 50.0, 2000), "mixed_orders": (W.mixed_orders_toy(), 6.0, 1500),
                      "oscillator": (W.vilar_oscillator(), 1.0, 600)}[case]
    theta = torch.tensor(spec.log_rates.astype(np.float32), device="cuda")
    ts = W.uniform_sample_grid(t_end, 11)
    obs = [0, 1] if spec.n_species > 1 else [0]
    net = S.Network(spec)
    dl = torch.tensor(W.seeded_dl_dobs(8, n, len(ts), len(obs), scale=1.0 / n), dtype=torch.float32, device="cuda")
    for specialize in (True, False):
        fw = S.forward(net, theta, n, spec.x0, t_end, ts, obs, 3, readout=readout, record=True, max_steps=1 << 16,
                       specialize=specialize, threads_per_traj=1)
        assert fw.run.variant == (2 if specialize else 1)
        for temps in ((0.1, 0.5, 1.0), (0.3, 2.0), (0.1, 0.5, 1.0, 0.05)):
            multi = S.backward_multi(fw, dl, temps)
            for t, T in enumerate(temps):
                one = S.backward(fw, dl, T)
                if specialize:
                    err = (multi[t] - one).abs().max().item()
                    assert err <= 1e-5 * one.abs().max().item(), (temps, t, multi[t], one)
                else:
                    assert torch.equal(multi[t], one), (temps, t, multi[t], one)
        _, mism = fw.run.status_counts()
        assert mism == 0
