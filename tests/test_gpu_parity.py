"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Parity levels for this method:
* Philox words: bit-exact.
* Integer states given the same event sequence (replay of the oracle's events): bit-exact.
* Event sequences: identical on >= 99.9% of trajectories; at the first step where a trajectory
  differs, the oracle's selection margin (s1 - s2)/s1 must be below 1e-6 (an FP32 key rounding).
* Observables on identical trajectories: HOLD exact, except samples within the clock tolerance of
  an event time; LINEAR within the interpolation error that the FP32 waiting times allow.
* Gradients: within 1e-3 relative (norm-wise) of the oracle's FP64 straight-through gradient.
* Forward law: ensemble moments within 3 standard errors of the exact master equation.
"""
import json
import os

import numpy as np
import pytest
import torch

import ssa_workloads as W
from ssa_workloads.configs import HOLD, LINEAR
from oracle import native

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
EPS32 = 2.0 ** -24
MARGIN_TOL = 1e-6
GRAD_RTOL = 1e-3


@pytest.fixture(scope="module")
def S():
    from paper_2602_19775_gb300 import ssa
    ssa._lib.lib()
    return ssa


def _oracle_theta(t32):
    """The log-rates the oracle receives for the binary32 parameters t32. The kernels form k = exp(theta) in
    binary64 and round it once to binary32: a relative error of up to 2^-24 that is the same at every step, so
    over ~1e6 draws it moves a trajectory's clock systematically (by ~1e-5 on the oscillator at t = 400). The
    oracle therefore gets the logarithm of those binary32 rate constants (as it gets the bf16 weights of the
    GRN), and both sides simulate the same rates; the gradient is d/dlog k at the same k on both."""
    k32 = np.exp(np.asarray(t32, dtype=np.float32).astype(np.float64)).astype(np.float32)
    return np.log(k32.astype(np.float64))


def _theta32(theta):
    """Parameters as the GPU receives them (binary32) and as the oracle receives the same rate constants."""
    t32 = np.asarray(theta, dtype=np.float32)
    return t32, _oracle_theta(t32)


def _run_both(S, net, theta, x0, n, t_end, ts, obs_sp, seed, readout, max_steps=4096, dl=None, T=1.0,
              K=64, traj_offset=0, ev_cap=None):
    t32, t64 = _theta32(theta)
    snet = S.Network(net)
    fw = S.forward(snet, torch.tensor(t32, device="cuda"), n, x0, t_end, ts, obs_sp, seed,
                   readout="hold" if readout == HOLD else "linear", record=True, ckpt_interval=K,
                   max_steps=max_steps, traj_offset=traj_offset)
    torch.cuda.synchronize()
    cap = ev_cap or max_steps
    orc = native.run(net, t64, x0, n, t_end, ts, obs_sp, seed, readout, max_steps=max_steps, traj_offset=traj_offset,
                     dl_dobs=dl, temperature=T, ev_cap=cap)
    gpu_ev = fw.run.events(cap).cpu().numpy()
    return snet, fw, orc, gpu_ev


def _divergence_rule(gpu_ev, draws_g, orc, crossing=None):
    """Event-sequence parity for trajectories of any length. Returns the mask of trajectories whose
    event sequences (and draw counts) agree with the oracle's, and asserts:
    (i) at the first step where a trajectory differs, the oracle's selection margin (s1 - s2)/s1 is below
        1e-6 (binary32 keys carry a few ulp), or `crossing(i, k)` says the divergence is a crossing
        decision within the clock tolerance of t_end;
    (ii) the number of trajectories that first differ at a near-tie is at most the oracle's own count of
        steps with margin below 1e-6 over all trajectories: with ~1e6 draws per trajectory a few flips are
        expected, so a floor on the identical fraction cannot hold, but each flip needs a near-tie."""
    draws_g = np.asarray(draws_g).astype(np.int64)
    same = np.all(gpu_ev == orc.events, axis=1) & (draws_g == orc.draws)
    n_tie = 0
    for i in np.nonzero(~same)[0]:
        diff = np.nonzero(gpu_ev[i] != orc.events[i])[0]
        k = int(diff[0]) if diff.size else int(min(draws_g[i], orc.draws[i]))
        m = orc.margins[i, k] if k < orc.draws[i] else 0.0
        if m < MARGIN_TOL:
            n_tie += 1
        else:
            assert crossing is not None and crossing(i, k), (i, k, m)
    steps = np.arange(orc.margins.shape[1])[None, :] < orc.draws[:, None]
    n_small = int(np.count_nonzero((orc.margins < MARGIN_TOL) & steps))
    assert n_tie <= n_small, (n_tie, n_small)
    return same


def _compare_events(orc, fw, gpu_ev, t_end, M, floor=0.999):
    """`_divergence_rule` with the crossing decision at t_end (network of M reactions); `floor` is the
    fraction of identical trajectories required of short trajectories (a few hundred draws; None for
    long ones, where the count rule (ii) alone applies)."""
    same = _divergence_rule(gpu_ev, fw.draws.cpu().numpy(), orc,
                            crossing=lambda i, k: _near_crossing(orc, i, k, t_end, M))
    if floor is not None:
        assert same.mean() >= floor, same.mean()
    return same


def _clock_tol(M, t):
    """Bound on |t_gpu - t_oracle| at time t: each binary32 waiting time tau = E_0/a0 carries at most
    ~(M + 2) unit roundoffs (a0 summed over M terms, the logarithm, the division), and the FP64 clock
    adds them up, so the drift is below (M + 2) u t; a factor 8 covers the 1-ulp logarithm."""
    return 8.0 * (M + 2) * EPS32 * np.asarray(t)


def _near_crossing(orc, i, k, t_end, M):
    """Whether draw k of trajectory i is the crossing of t_end within the clock tolerance."""
    t = orc.times[i, k] if k < orc.times.shape[1] else np.nan
    return bool(np.isfinite(t) and abs(t - t_end) <= _clock_tol(M, t_end))


def _oracle_brackets(orc, ts):
    """Index k of the state with t_k <= t_s < t_{k+1}, from the oracle's event times."""
    n = orc.draws.shape[0]
    out = np.zeros((n, len(ts)), dtype=np.int64)
    for i in range(n):
        d = int(orc.draws[i])
        applied = d - 1 if orc.status[i] in (native.STATUS["OK"], native.STATUS["NEG_COUNT"],
                                             native.STATUS["OVERFLOW"]) else d
        out[i] = np.searchsorted(orc.times[i, :applied], ts, side="right")
    return out


def _bracket_agreement(orc, fw, ts, M):
    """Trajectories whose sample brackets agree with the oracle's. A flip is only allowed where an
    event time lies within the FP32 clock tolerance of the sample time; the LINEAR readout's time
    derivative jumps there (the interpolation slope changes at an event), so such a trajectory's
    gradient is not comparable and it is left out of the gradient parity."""
    gb = fw.run.brackets().cpu().numpy()
    ob = _oracle_brackets(orc, ts)
    agree = np.all(gb == ob, axis=1)
    for i in np.nonzero(~agree)[0]:
        for s in np.nonzero(gb[i] != ob[i])[0]:
            ev_t = orc.times[i, :orc.draws[i]]
            assert np.min(np.abs(ev_t - ts[s])) <= _clock_tol(M, ts[s]), (i, s)
    return agree


def _bracket_flips(orc, fw, ts, M):
    """[n, S] mask of the samples whose bracket differs from the oracle's, each checked to lie within the
    clock tolerance of an event time. Over ~1e6 draws the binary32 waiting times move the clock by more
    than the spacing of events, so most long trajectories flip a few of their samples; the gradient is
    linear in dL/dobs, so zeroing the upstream gradient of exactly those samples on both sides compares
    everything else."""
    gb = fw.run.brackets().cpu().numpy()
    ob = _oracle_brackets(orc, ts)
    flip = gb != ob
    for i, s in zip(*np.nonzero(flip)):
        ev_t = orc.times[i, :orc.draws[i]]
        assert np.min(np.abs(ev_t - ts[s])) <= _clock_tol(M, ts[s]), (i, s)
    return flip


def test_philox_words_bit_exact(S):
    rng = np.random.default_rng(0)
    traj = rng.integers(0, 2 ** 40, size=257)
    step = rng.integers(0, 2 ** 31, size=257)
    seed = 0xDEADBEEF12345678
    g = S.philox_uniforms(seed, traj, step, 13).cpu().numpy().astype(np.float64)
    ref = np.stack([native.uniforms(seed, int(a), int(b), 13) for a, b in zip(traj, step)])
    np.testing.assert_array_equal(g, ref)


def test_forward_c1_matches_oracle(S):
    wl = W.config_c1()
    snet, fw, orc, gpu_ev = _run_both(S, wl.net, wl.log_rates, wl.x0, wl.n_traj, wl.t_end, wl.sample_times,
                                      wl.obs_species, wl.seed, HOLD)
    st = fw.status.cpu().numpy()
    assert np.all(st == 0)
    same = _compare_events(orc, fw, gpu_ev, wl.t_end, wl.net.n_reactions)
    obs_g = fw.obs.cpu().numpy()
    for i in np.nonzero(same)[0]:
        d = np.nonzero(np.any(obs_g[i] != orc.obs[i], axis=1))[0]
        for s in d:  # only where an event lies within the clock tolerance of the sample time
            ts = wl.sample_times[s]
            assert np.min(np.abs(orc.times[i, :orc.draws[i]] - ts)) <= _clock_tol(2, ts), (i, s)


def test_forward_moments_match_exact_cme(S):
    gold = json.load(open(os.path.join(GOLDEN, "dimer_2a_b_cme.json")))
    wl = W.config_c1(n_traj=65536)
    snet = S.Network(wl.net)
    fw = S.forward(snet, torch.tensor(wl.log_rates.astype(np.float32), device="cuda"), wl.n_traj, wl.x0, wl.t_end,
                   wl.sample_times, wl.obs_species, 7, readout="hold", max_steps=4096)
    A = fw.obs[:, :, 0].double().cpu().numpy()
    B = fw.obs[:, :, 1].double().cpu().numpy()
    np.testing.assert_array_equal(A + 2 * B, 100)
    m = A.mean(0)
    se = A.std(0, ddof=1) / np.sqrt(A.shape[0])
    z = (m - np.array(gold["mean_A"])) / se
    assert np.all(np.abs(z) < 3.0), z
    v = A.var(0, ddof=1)
    mu4 = ((A - m) ** 4).mean(0)
    zv = (v - np.array(gold["var_A"])) / np.sqrt((mu4 - v ** 2) / A.shape[0])
    assert np.all(np.abs(zv) < 3.0), zv


@pytest.mark.parametrize("readout", [HOLD, LINEAR])
def test_replay_oracle_events_bit_exact_states(S, readout):
    net = W.mixed_orders_toy()
    n, t_end = 777, 6.0
    ts = W.uniform_sample_grid(t_end, 13)
    obs_sp = np.array([0, 1, 2], np.int32)
    t32, t64 = _theta32(net.log_rates)
    cap = 2048
    orc = native.run(net, t64, net.x0, n, t_end, ts, obs_sp, 3, readout, max_steps=cap, ev_cap=cap)
    snet = S.Network(net)
    ev = np.where(orc.events >= 0, orc.events, 0).astype(np.int32)
    nev = orc.draws.astype(np.int32)
    fw = S.forward(snet, torch.tensor(t32, device="cuda"), n, net.x0, t_end, ts, obs_sp, 3,
                   readout="hold" if readout == HOLD else "linear", record=True, max_steps=cap,
                   replay_events=torch.tensor(ev, device="cuda"), replay_n_events=nev)
    st = fw.status.cpu().numpy()
    ok = st != 7
    assert ok.mean() > 0.99
    np.testing.assert_array_equal(fw.draws.cpu().numpy()[ok], orc.draws[ok])
    # the recorded log is the given sequence, and the reconstructed final states agree exactly
    gev = fw.run.events(cap).cpu().numpy()
    np.testing.assert_array_equal(gev[ok], orc.events[ok])
    obs_g = fw.obs.double().cpu().numpy()
    if readout == HOLD:
        diff = np.any(obs_g != orc.obs, axis=2) & ok[:, None]
        assert diff.mean() < 1e-3
    else:
        err = np.abs(obs_g - orc.obs)[ok]
        assert np.quantile(err, 0.999) < 1e-4


def _grad_case(S, net, theta, x0, n, t_end, ts, obs_sp, seed, readout, T, dl_seed=5, K=64, max_steps=4096):
    dl = W.seeded_dl_dobs(dl_seed, n, len(ts), len(obs_sp), scale=1.0 / n)
    snet, fw, orc, gpu_ev = _run_both(S, net, theta, x0, n, t_end, ts, obs_sp, seed, readout, max_steps=max_steps,
                                      dl=dl, T=T, K=K)
    same = _compare_events(orc, fw, gpu_ev, t_end, net.n_reactions)
    agree = _bracket_agreement(orc, fw, np.asarray(ts), net.n_reactions)
    assert agree.mean() >= 0.99, agree.mean()
    same &= agree
    # the GPU gradient is the sum over trajectories: zero the upstream gradient of any divergent one
    dl_g = dl.copy()
    dl_g[~same] = 0.0
    g = S.backward(fw, torch.tensor(dl_g, dtype=torch.float32, device="cuda"), T).cpu().numpy().astype(np.float64)
    ref = orc.dtheta[same].sum(0)
    counts, mism = fw.run.status_counts()
    assert mism == 0, mism
    rel = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30)
    assert rel < GRAD_RTOL, (rel, g, ref)
    big = np.abs(ref) > 1e-3 * np.linalg.norm(ref)
    np.testing.assert_allclose(g[big], ref[big], rtol=2 * GRAD_RTOL)
    return rel


@pytest.mark.parametrize("T", [0.1, 0.5, 1.0])
def test_backward_c2_matches_oracle(S, T):
    wl = W.config_c2(n_traj=4096)
    _grad_case(S, wl.net, wl.log_rates, wl.x0, wl.n_traj, wl.t_end, wl.sample_times, wl.obs_species, wl.seed,
               LINEAR, T)


@pytest.mark.parametrize("readout", [HOLD, LINEAR])
def test_backward_mixed_orders_matches_oracle(S, readout):
    net = W.mixed_orders_toy()
    ts = W.uniform_sample_grid(6.0, 11)
    _grad_case(S, net, net.log_rates, net.x0, 1000, 6.0, ts, np.array([0, 1, 2], np.int32), 9, readout, 0.5, K=16)


def test_backward_oscillator_short_matches_oracle(S):
    net = W.vilar_oscillator()
    ts = W.uniform_sample_grid(2.0, 20)
    _grad_case(S, net, net.log_rates, net.x0, 512, 2.0, ts, np.array([6, 7, 8], np.int32), 4, LINEAR, 0.3,
               max_steps=1 << 15)


def test_backward_replay_all_trajectories(S):
    """Replay the oracle's events, so that every trajectory is compared, divergences included."""
    wl = W.config_c2(n_traj=2048)
    n = wl.n_traj
    t32, t64 = _theta32(wl.log_rates)
    dl = W.seeded_dl_dobs(17, n, len(wl.sample_times), 1, scale=1.0 / n)
    cap = 4096
    orc = native.run(wl.net, t64, wl.x0, n, wl.t_end, wl.sample_times, wl.obs_species, 11, LINEAR, max_steps=cap,
                     dl_dobs=dl, temperature=0.5, ev_cap=cap)
    snet = S.Network(wl.net)
    ev = np.where(orc.events >= 0, orc.events, 0).astype(np.int32)
    fw = S.forward(snet, torch.tensor(t32, device="cuda"), n, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, 11,
                   readout="linear", record=True, max_steps=cap, replay_events=torch.tensor(ev, device="cuda"),
                   replay_n_events=orc.draws.astype(np.int32))
    ok = fw.status.cpu().numpy() == 0
    assert ok.mean() > 0.99
    dl_g = dl.copy()
    dl_g[~ok] = 0
    g = S.backward(fw, torch.tensor(dl_g, dtype=torch.float32, device="cuda"), 0.5).cpu().numpy()
    ref = orc.dtheta[ok].sum(0)
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel < GRAD_RTOL, (rel, g, ref)


def test_conserved_quantity_gradient_vanishes(S):
    wl = W.config_c2(n_traj=1024)
    snet = S.Network(wl.net)
    fw = S.forward(snet, torch.tensor(wl.log_rates.astype(np.float32), device="cuda"), wl.n_traj, wl.x0, wl.t_end,
                   wl.sample_times, [0, 1], 2, readout="linear", record=True)
    dl = torch.zeros((wl.n_traj, len(wl.sample_times), 2), device="cuda")
    dl[:, :, 0] = 1.0
    dl[:, :, 1] = 2.0
    g = S.backward(fw, dl, 0.5).cpu().numpy()
    # cancellation is exact in the surrogate; FP32 rounding leaves ~1e-6 of the per-term scale
    assert np.abs(g).max() < 1e-3 * wl.n_traj * len(wl.sample_times) * 1e-3


def test_autograd_function_matches_backward(S):
    wl = W.config_c2(n_traj=512)
    snet = S.Network(wl.net)
    theta = torch.tensor(wl.log_rates.astype(np.float32), device="cuda", requires_grad=True)
    obs = S.simulate(snet, theta, wl.n_traj, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, 0,
                     readout="linear", temperature=0.5)
    target = torch.linspace(90, 30, len(wl.sample_times), device="cuda")
    loss = ((obs[:, :, 0].mean(0) - target) ** 2).mean()
    loss.backward()
    fw = S.forward(snet, theta.detach(), wl.n_traj, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, 0,
                   readout="linear", record=True)
    m = fw.obs[:, :, 0].mean(0)
    dl = (2.0 * (m - target) / len(wl.sample_times) / wl.n_traj)[None, :, None].expand(wl.n_traj, -1, 1)
    g = S.backward(fw, dl.contiguous(), 0.5)
    torch.testing.assert_close(theta.grad, g, rtol=1e-5, atol=1e-7)


def test_ensemble_mean_matches_torch(S):
    x = torch.randint(0, 1000, (70001, 37), dtype=torch.int32, device="cuda")
    m = S.ensemble_mean(x)
    torch.testing.assert_close(m, x.double().mean(0).float(), rtol=1e-5, atol=1e-4)
    y = torch.randn((3001, 5, 3), device="cuda")
    torch.testing.assert_close(S.ensemble_mean(y), y.mean(0), rtol=1e-4, atol=1e-5)
    # bitwise reproducible
    assert torch.equal(S.ensemble_mean(y), S.ensemble_mean(y))


def test_determinism_and_chunking_invariance(S):
    wl = W.config_c2(n_traj=3000)
    snet = S.Network(wl.net)
    th = torch.tensor(wl.log_rates.astype(np.float32), device="cuda")
    a = S.forward(snet, th, 3000, wl.x0, wl.t_end, wl.sample_times, [0, 1], 5, readout="linear", record=True)
    b = S.forward(snet, th, 3000, wl.x0, wl.t_end, wl.sample_times, [0, 1], 5, readout="linear", record=True,
                  block_threads=64)
    c1 = S.forward(snet, th, 1234, wl.x0, wl.t_end, wl.sample_times, [0, 1], 5, readout="linear")
    c2 = S.forward(snet, th, 3000 - 1234, wl.x0, wl.t_end, wl.sample_times, [0, 1], 5, readout="linear",
                   traj_offset=1234)
    assert torch.equal(a.obs, b.obs)
    assert torch.equal(a.obs, torch.cat([c1.obs, c2.obs]))
    dl = torch.randn_like(a.obs) / 3000
    ga = S.backward(a, dl, 0.5)
    gb = S.backward(b, dl, 0.5)
    ga2 = S.backward(a, dl, 0.5)
    assert torch.equal(ga, ga2)
    torch.testing.assert_close(ga, gb, rtol=1e-5, atol=1e-6)


def test_edge_cases(S):
    net = W.dimerization_2a_b()
    snet = S.Network(net)
    th = torch.tensor(net.log_rates.astype(np.float32), device="cuda")
    ts = np.array([0.0, 1.0, 2.0])
    # empty batch
    r = S.forward(snet, th, 0, net.x0, 2.0, ts, [0], 0, record=True)
    assert r.obs.shape == (0, 3, 1)
    assert torch.equal(S.backward(r, torch.zeros((0, 3, 1), device="cuda"), 1.0), torch.zeros(2, device="cuda"))
    # one trajectory, ragged batch sizes
    for n in (1, 33, 129, 1000):
        r = S.forward(snet, th, n, net.x0, 2.0, ts, [0], 0, record=True)
        o = native.run(net, net.log_rates.astype(np.float32).astype(np.float64), net.x0, n, 2.0, ts,
                       np.array([0], np.int32), 0, HOLD)
        assert np.mean(np.all(r.obs.cpu().numpy() == o.obs, axis=(1, 2))) > 0.99
    # t_end = 0: one crossing draw, state holds
    r = S.forward(snet, th, 5, net.x0, 0.0, [0.0], [0], 0, readout="linear")
    assert torch.all(r.draws == 1) and torch.all(r.obs == 100)
    # absorbing from the start (A = 1, B = 0)
    r = S.forward(snet, th, 5, np.array([1, 0], np.int32), 2.0, ts, [0], 0, readout="linear", record=True)
    assert torch.all(r.status == 1) and torch.all(r.draws == 0) and torch.all(r.obs == 1)
    g = S.backward(r, torch.ones((5, 3, 1), device="cuda"), 1.0)
    assert torch.all(g == 0)
    # step cap
    r = S.forward(snet, th, 5, net.x0, 1e9, ts, [0], 0, max_steps=7, record=True)
    assert torch.all(r.status == 2) and torch.all(r.draws == 7)
    # invalid sample times and observed species are reported per trajectory, never read out of bounds
    r = S.forward(snet, th, 4, net.x0, 1.0, [0.5, 0.2], [0], 0)
    assert torch.all(r.status == 6)
    r = S.forward(snet, th, 4, net.x0, 1.0, [0.5], [5], 0)
    assert torch.all(r.status == 6)
    # argument errors come back as exceptions, not faults
    from paper_2602_19775_gb300 import SSAError
    with pytest.raises(SSAError):
        S.forward(snet, th, 4, net.x0, -1.0, ts, [0], 0)
    with pytest.raises(SSAError):
        S.backward(S.forward(snet, th, 4, net.x0, 1.0, [0.5], [0], 0), torch.zeros((4, 1, 1), device="cuda"), 1.0)
