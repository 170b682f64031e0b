"""GPU tests of the network-specialised kernels (compiled at run time for one network): they reproduce
the generic thread-per-trajectory kernels bit for bit -- observables, draws, status codes, event logs,
sample brackets -- and their gradients to binary32 rounding, on networks covering every mass-action
order, the HOLD, LINEAR and BIN readouts, and the size limits; networks above the limits keep the generic
kernels. Parity of the specialised kernels with the FP64 oracle is covered by the oracle tests, which
run them by default."""
import numpy as np
import pytest
import torch

import ssa_workloads as W

from test_gpu_warp import _pilot_t_end

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2602_19775_gb300 import ssa
    ssa._lib.lib()
    return ssa


def _random(seed, n_sp, n_rx):
    return W.random_network(np.random.default_rng(seed), n_species_range=n_sp, n_reactions_range=n_rx)


CASES = {
    "dimer": lambda: (W.dimerization_2a_b(), 50.0, [0, 1]),
    "immigration_death": lambda: (W.immigration_death(), 5.0, [0]),
    "ion_channel": lambda: (W.ion_channel_coi(), 8.0, [1]),
    "mixed_orders": lambda: (W.mixed_orders_toy(), 6.0, [0, 1, 2]),
    "oscillator": lambda: (W.vilar_oscillator(), 1.0, [6, 7, 8]),
    "random_10": lambda: (_random(21, (3, 8), (10, 10)), None, [0, 1]),
    "random_24": lambda: (_random(7, (10, 24), (24, 24)), None, [0, 1, 2]),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("readout", ["hold", "linear", "bin"])
def test_specialised_kernels_match_generic(S, case, readout):
    spec, t_end, obs = CASES[case]()
    if t_end is None:
        t_end = _pilot_t_end(spec, spec.log_rates.astype(np.float32).astype(np.float64))
    net = S.Network(spec)
    ok, why = net.specialize()
    assert ok, why
    theta = torch.tensor(spec.log_rates.astype(np.float32), device="cuda")
    ts = W.uniform_sample_grid(t_end, 12)
    n, cap = 1000, 1 << 14
    runs = []
    for specialize in (True, False):
        fw = S.forward(net, theta, n, spec.x0, t_end, ts, obs, 5, readout=readout, record=True, max_steps=cap,
                       threads_per_traj=1, specialize=specialize, traj_offset=3)
        runs.append(fw)
    a, b = runs
    assert a.run.variant == 2 and b.run.variant == 1
    assert torch.equal(a.obs, b.obs)
    assert torch.equal(a.draws, b.draws) and torch.equal(a.status, b.status)
    assert torch.equal(a.run.events(cap), b.run.events(cap))
    assert torch.equal(a.run.brackets(), b.run.brackets())
    dl = torch.tensor(W.seeded_dl_dobs(9, n, len(ts), len(obs), scale=1.0 / n), dtype=torch.float32, device="cuda")
    for T in (0.1, 1.0):
        ga = S.backward(a, dl, T).double().cpu().numpy()
        gb = S.backward(b, dl, T).double().cpu().numpy()
        assert a.run.status_counts()[1] == 0 and b.run.status_counts()[1] == 0
        scale = max(np.abs(gb).max(), 1e-30)
        assert np.abs(ga - gb).max() <= 1e-5 * scale, (T, np.abs(ga - gb).max(), scale)


def test_networks_above_the_limits_keep_the_generic_kernels(S):
    spec = _random(5, (6, 12), (30, 30))
    net = S.Network(spec)
    ok, why = net.specialize()
    assert not ok and "limits" in why
    fw = S.forward(net, torch.tensor(spec.log_rates.astype(np.float32), device="cuda"), 64, spec.x0, 0.01, [0.01],
                   [0], 1, record=True, threads_per_traj=1, max_steps=4096)
    assert fw.run.variant == 1


def test_default_choice_uses_the_specialised_kernels(S):
    wl = W.config_c2(n_traj=256)
    net = S.Network(wl.net)
    fw = S.forward(net, torch.tensor(wl.log_rates.astype(np.float32), device="cuda"), 256, wl.x0, wl.t_end,
                   wl.sample_times, wl.obs_species, 0, readout="linear", record=True, max_steps=4096)
    assert fw.run.variant == 2


@pytest.mark.parametrize("case", ["dimer", "mixed_orders", "oscillator"])
def test_direct_method_matches_oracle(S, case):
    """The plain direct method (u_1 a0 against the cumulative propensities) against the FP64 oracle's
    direct method on the same uniforms: identical draw counts and HOLD observables on all but a few
    trajectories (a choice can flip only where u_1 a0 lies within binary32 rounding of a cumulative
    boundary)."""
    from oracle import native
    spec, t_end, obs = CASES[case]()
    net = S.Network(spec)
    theta32 = spec.log_rates.astype(np.float32)
    ts = W.uniform_sample_grid(t_end, 10)
    n = 2000
    fw = S.forward(net, torch.tensor(theta32, device="cuda"), n, spec.x0, t_end, ts, obs, 21, readout="hold",
                   max_steps=1 << 15, selector="direct", traj_offset=5)
    assert fw.run.variant == 2
    orc = native.run(spec, theta32.astype(np.float64), spec.x0, n, t_end, ts, np.array(obs, np.int32), 21,
                     native.HOLD, max_steps=1 << 15, traj_offset=5, selector="direct")
    np.testing.assert_array_equal(fw.status.cpu().numpy(), orc.status)
    same = (fw.draws.cpu().numpy() == orc.draws) & np.all(fw.obs.cpu().numpy() == orc.obs, axis=(1, 2))
    assert same.mean() >= 0.99, same.mean()


def test_direct_method_moments_match_exact_cme(S):
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dimer_2a_b_cme.json")))
    wl = W.config_c1(n_traj=65536)
    net = S.Network(wl.net)
    fw = S.forward(net, torch.tensor(wl.log_rates.astype(np.float32), device="cuda"), wl.n_traj, wl.x0, wl.t_end,
                   wl.sample_times, wl.obs_species, 0, readout="hold", max_steps=4096, selector="direct")
    A = fw.obs[:, :, 0].double().cpu().numpy()
    m = A.mean(0)
    se = A.std(0, ddof=1) / np.sqrt(wl.n_traj)
    z = (m - np.array(gold["mean_A"])) / se
    assert np.all(np.abs(z) < 3.5), z  # 50 sample times at once


def test_direct_method_is_forward_only(S):
    from paper_2602_19775_gb300 import SSAError
    spec = W.dimerization_2a_b()
    net = S.Network(spec)
    with pytest.raises(SSAError):
        S.forward(net, torch.tensor(spec.log_rates.astype(np.float32), device="cuda"), 8, spec.x0, 1.0, [1.0], [0],
                  0, record=True, selector="direct")


@pytest.mark.parametrize("readout", ["hold", "linear"])
@pytest.mark.parametrize("record", [False, True])
def test_staged_sample_stores_match_direct_stores(S, readout, record):
    """The specialised forward collects each thread's samples in windows and copies completed windows warp-wide;
    the observables must be those of the generic kernels' direct stores bit for bit: dense grids where
    several windows complete within one step, 1 to 4 observables (5 is stored directly), paths that absorb
    early (the held tail), and a partial last warp."""
    cases = [
        (W.immigration_death(), 5.0, 2003, [0]),                       # ~100 samples per event
        (W.mixed_orders_toy(), 6.0, 997, [0, 1]),
        (W.mixed_orders_toy(), 6.0, 333, [2, 0, 1]),
        (W.vilar_oscillator(), 0.5, 129, [6, 7, 8, 0]),
        (W.vilar_oscillator(), 0.5, 77, [6, 7, 8, 0, 1]),              # n_obs = 5: direct stores
        (W.network_from_reactions(["A"], [(["A"], [], "d")], {"d": 2.0}, {"A": 20}), 30.0, 600, [0]),  # absorbs
    ]
    for spec, t_end, n_s, obs in cases:
        net = S.Network(spec)
        theta = torch.tensor(spec.log_rates.astype(np.float32), device="cuda")
        ts = W.uniform_sample_grid(t_end, n_s)
        n = 1000
        runs = [S.forward(net, theta, n, spec.x0, t_end, ts, obs, 11, readout=readout, record=record, max_steps=1 << 16,
                          threads_per_traj=1, specialize=sp) for sp in (True, False)]
        assert runs[0].run.variant == 2 and runs[1].run.variant == 1
        assert torch.equal(runs[0].obs, runs[1].obs), (spec.species, n_s, obs)
        assert torch.equal(runs[0].draws, runs[1].draws)
        if record:
            assert torch.equal(runs[0].run.brackets(), runs[1].run.brackets())
