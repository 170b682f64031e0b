"""GPU tests of the batch of networks (one persistent forward and one persistent adjoint launch for
many networks of different sizes): each item reproduces the single-network entry points bit for bit
in its observables, draws and status codes, and to binary32 summation order in its gradient; the
gradient bits do not depend on which warp ran which work unit; a captured CUDA graph replays the
same computation with updated parameters; the pilot autotuner picks a valid plan."""
import numpy as np
import pytest
import torch

import ssa_workloads as W
from ssa_workloads.configs import LINEAR

from test_gpu_warp import _pilot_t_end

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2602_19775_gb300 import ssa
    ssa._lib.lib()
    return ssa


def _random(seed, n_sp, n_rx):
    return W.random_network(np.random.default_rng(seed), n_species_range=n_sp, n_reactions_range=n_rx)


@pytest.fixture(scope="module")
def specs():
    """(network, n_traj, t_end, n_samples, obs species, seed, threads_per_traj, max_steps) per item."""
    dimer = W.dimerization_2a_b()
    imm = W.immigration_death()
    osc = W.vilar_oscillator()
    r10 = _random(21, (3, 8), (10, 10))
    r_big = _random(3, (8, 64), (100, 200))
    r30 = _random(5, (6, 12), (20, 40))
    out = [
        (dimer, 300, 20.0, 10, [0, 1], 11, 0, 4096),
        (imm, 33, 5.0, 5, [0], 12, 0, 4096),
        (osc, 64, 1.0, 8, [6, 7, 8], 13, 0, 1 << 14),
        (r10, 70, None, 6, [0, 1], 14, 0, 4096),
        (r_big, 9, None, 6, [0, 1, 2], 15, 0, 4096),
        (r30, 20, None, 6, [0, 1], 16, 32, 4096),
        (dimer, 0, 20.0, 4, [0], 17, 0, 4096),
    ]
    res = []
    for net, n, t_end, ns, obs, seed, tpt, ms in out:
        if t_end is None:
            t_end = _pilot_t_end(net, net.log_rates.astype(np.float32).astype(np.float64))
        res.append((net, n, t_end, ns, obs, seed, tpt, ms))
    return res


def _items(S, specs, nets, theta_shift=0.0):
    items = []
    for q, (net, n, t_end, ns, obs, seed, tpt, ms) in enumerate(specs):
        items.append(dict(net=nets[q], log_rates=(net.log_rates + theta_shift).astype(np.float32), n_traj=n,
                          x0=net.x0, t_end=t_end, sample_times=W.uniform_sample_grid(t_end, ns), obs_species=obs,
                          seed=seed, traj_offset=7 * q, max_steps=ms, threads_per_traj=tpt, ckpt_interval=64))
    return items


def _fill_dl(b, specs, seed=3):
    for q, (net, n, t_end, ns, obs, *_rest) in enumerate(specs):
        dl = W.seeded_dl_dobs(seed + q, n, ns, len(obs), scale=1.0 / max(n, 1))
        b.dl_dobs[q].copy_(torch.tensor(dl, dtype=torch.float32))


def _single(S, net, item, variant, dl, T, readout="linear"):
    fw = S.forward(net, torch.tensor(item["log_rates"], device="cuda"), item["n_traj"], item["x0"], item["t_end"],
                   item["sample_times"], item["obs_species"], item["seed"], readout=readout, record=True,
                   max_steps=item["max_steps"], traj_offset=item["traj_offset"], threads_per_traj=variant,
                   ckpt_interval=64)
    g = S.backward(fw, dl, T) if item["n_traj"] > 0 else torch.zeros(net.n_params, device="cuda")
    return fw, g


def _check_against_single(S, b, specs, nets, items, T, readout="linear"):
    for q in range(len(specs)):
        v = b.variant(q)
        assert v in (1, 32)
        fw, g = _single(S, nets[q], items[q], v, b.dl_dobs[q], T, readout)
        draws, status, mism = b.outputs(q)
        assert mism == 0
        torch.testing.assert_close(b.obs[q], fw.obs, rtol=0, atol=0)
        assert torch.equal(draws, fw.draws) and torch.equal(status, fw.status)
        assert torch.all(status <= 2), q  # OK, ABSORBED or STEP_CAP
        gb, gs = b.dtheta[q].double().cpu().numpy(), g.double().cpu().numpy()
        scale = max(np.abs(gs).max(), 1e-12)
        assert np.abs(gb - gs).max() <= 1e-4 * scale, (q, np.abs(gb - gs).max(), scale)


def test_batch_matches_single_network_entry_points(S, specs):
    nets = [S.Network(s[0]) for s in specs]
    items = _items(S, specs, nets)
    b = S.Batch(items, readout="linear", temperature=0.5)
    assert [b.variant(q) for q in range(len(specs))] == [1, 1, 1, 1, 32, 32, 1]
    _fill_dl(b, specs)
    b.run()
    _check_against_single(S, b, specs, nets, items, 0.5)
    assert torch.all(b.dtheta[6] == 0)


def test_batch_gradient_bits_do_not_depend_on_unit_order(S, specs):
    nets = [S.Network(s[0]) for s in specs]
    b = S.Batch(_items(S, specs, nets), readout="linear", temperature=0.5)
    _fill_dl(b, specs)
    b.run()
    first = [t.clone() for t in b.dtheta]
    for _ in range(3):
        b.run()
        for q in range(len(specs)):
            assert torch.equal(b.dtheta[q], first[q]), q


def test_batch_graph_replay_with_updated_parameters(S, specs):
    nets = [S.Network(s[0]) for s in specs]
    stream = torch.cuda.Stream()
    g = S.Batch(_items(S, specs, nets), readout="linear", temperature=0.5)
    _fill_dl(g, specs)
    with torch.cuda.stream(stream):
        g.run(use_graph=True, stream=stream)
    stream.synchronize()
    ref = S.Batch(_items(S, specs, nets), readout="linear", temperature=0.5)
    _fill_dl(ref, specs)
    ref.run()
    torch.cuda.synchronize()
    for q in range(len(specs)):
        assert torch.equal(g.obs[q], ref.obs[q]) and torch.equal(g.dtheta[q], ref.dtheta[q]), q
    # new parameters and upstream gradients written in place, graph replayed
    items2 = _items(S, specs, nets, theta_shift=0.05)
    for q in range(len(specs)):
        g.log_rates[q].copy_(torch.tensor(items2[q]["log_rates"]))
    _fill_dl(g, specs, seed=40)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        g.run(use_graph=True, stream=stream)
    stream.synchronize()
    ref2 = S.Batch(items2, readout="linear", temperature=0.5)
    _fill_dl(ref2, specs, seed=40)
    ref2.run()
    torch.cuda.synchronize()
    for q in range(len(specs)):
        assert torch.equal(g.obs[q], ref2.obs[q]) and torch.equal(g.dtheta[q], ref2.dtheta[q]), q
    assert not torch.equal(g.obs[0], ref.obs[0])


def test_batch_autotune_plan_is_valid_and_exact(S, specs):
    nets = [S.Network(s[0]) for s in specs]
    items = _items(S, specs, nets)
    b = S.Batch(items, readout="linear", temperature=0.7)
    draws = b.autotune(pilot_traj=32)
    assert all(d >= 1.0 for d in draws)
    assert b.variant(5) == 32  # requested explicitly
    # the checkpoint interval: c x 16 N for one of the three timed scales, or the item's own
    for q, (spec, *_rest) in enumerate(specs):
        K = b.ckpt_interval(q)
        fixed = items[q].get("ckpt_interval", 0)
        if fixed:
            assert K == fixed
        else:
            base = min(1024, max(16, (16 * spec.n_species + 7) // 8 * 8))
            assert K % 8 == 0 and 8 <= K <= 4096
            assert K in {min(4096, max(8, int(c * base / 8.0 + 0.5) * 8)) for c in (0.25, 1.0, 4.0)}, (q, K)
    _fill_dl(b, specs)
    b.run()
    _check_against_single(S, b, specs, nets, items, 0.7)


def test_batch_item_with_bad_samples_is_isolated(S):
    dimer = W.dimerization_2a_b()
    net = S.Network(dimer)
    ok = dict(net=net, log_rates=dimer.log_rates.astype(np.float32), n_traj=40, x0=dimer.x0, t_end=10.0,
              sample_times=W.uniform_sample_grid(10.0, 5), obs_species=[0], seed=1)
    bad = dict(ok, sample_times=np.array([1.0, 3.0, 2.0]), seed=2)
    b = S.Batch([ok, bad], readout="hold", temperature=0.5)
    b.run()
    _, st_ok, _ = b.outputs(0)
    _, st_bad, _ = b.outputs(1)
    assert torch.all(st_ok == 0)
    assert torch.all(st_bad == 6)  # SSA_TRAJ_BAD_INPUT
    assert torch.all(b.dtheta[1] == 0)


def test_batch_rejects_invalid_items(S):
    from paper_2602_19775_gb300 import SSAError
    dimer = W.dimerization_2a_b()
    net = S.Network(dimer)
    base = dict(net=net, log_rates=dimer.log_rates.astype(np.float32), n_traj=8, x0=dimer.x0, t_end=1.0,
                sample_times=[0.5], obs_species=[0], seed=1)
    with pytest.raises(SSAError):
        S.Batch([dict(base, ckpt_interval=12)])
    with pytest.raises(SSAError):
        S.Batch([dict(base, max_steps=0)])
    big = S.Network(_random(3, (20, 30), (40, 60)))
    with pytest.raises(SSAError):
        S.Batch([dict(base, net=big, x0=np.zeros(big.n_species, np.int32), threads_per_traj=1)])


def test_batch_matches_oracle_on_uneven_random_networks(S):
    """Items of the uneven random-network workload (first draws of its seeded stream, trajectory counts
    scaled down to oracle size) against the FP64 oracle: status codes, event sequences under the margin
    rule, observables, and gradients on trajectories whose events and brackets agree."""
    from oracle import native
    from test_gpu_parity import GRAD_RTOL, _bracket_agreement, _clock_tol, _compare_events, _oracle_brackets
    from types import SimpleNamespace

    wl = W.config_c4(n_nets=5, traj_scale=1.0 / 256)
    cap = 1 << 15
    nets = [S.Network(spec) for spec in wl.nets]
    items = [dict(net=nets[q], log_rates=spec.log_rates.astype(np.float32), n_traj=int(wl.n_traj[q]), x0=spec.x0,
                  t_end=wl.t_end, sample_times=wl.sample_times, obs_species=wl.obs_species[q], seed=60 + q,
                  traj_offset=1000 * q, max_steps=cap) for q, spec in enumerate(wl.nets)]
    b = S.Batch(items, readout="linear", temperature=wl.temperature)
    dls = []
    for q in range(len(items)):
        dl = W.seeded_dl_dobs(80 + q, items[q]["n_traj"], len(wl.sample_times), len(wl.obs_species[q]),
                              scale=1.0 / items[q]["n_traj"])
        dls.append(dl)
        b.dl_dobs[q].copy_(torch.tensor(dl, dtype=torch.float32))
    b.run()
    torch.cuda.synchronize()
    for q, spec in enumerate(wl.nets):
        it = items[q]
        n = it["n_traj"]
        draws, status, mism = b.outputs(q)
        assert mism == 0
        orc = native.run(spec, spec.log_rates.astype(np.float32).astype(np.float64), spec.x0, n, wl.t_end,
                         wl.sample_times, wl.obs_species[q], it["seed"], LINEAR, max_steps=cap,
                         traj_offset=it["traj_offset"], dl_dobs=dls[q], temperature=wl.temperature, ev_cap=cap)
        np.testing.assert_array_equal(status.cpu().numpy(), orc.status)
        fw = SimpleNamespace(draws=draws, status=status,
                             run=SimpleNamespace(brackets=lambda q=q: b.brackets(q)))
        # thousands of draws per trajectory, up to 512 reactions: the count rule, and a floor of 0.9
        same = _compare_events(orc, fw, b.events(q, cap).cpu().numpy(), wl.t_end, spec.n_reactions, floor=0.9)
        agree = _bracket_agreement(orc, fw, wl.sample_times, spec.n_reactions)
        use = same & agree
        obs = b.obs[q].double().cpu().numpy()
        ob = _oracle_brackets(orc, wl.sample_times)
        vmax = np.abs(spec.stoich_delta).max()
        for i in np.nonzero(use)[0]:
            t = np.concatenate([[0.0], orc.times[i, :orc.draws[i]]])
            k = ob[i]
            tau = t[np.minimum(k + 1, len(t) - 1)] - t[k]
            tol = vmax * _clock_tol(spec.n_reactions, wl.sample_times) / np.maximum(tau, 1e-300) \
                + 1e-6 * np.abs(orc.obs[i]).max(1)
            assert np.all(np.abs(obs[i] - orc.obs[i]).max(1) <= tol), (q, i)
        # gradient over the agreeing trajectories: rerun the item alone with the others' upstream zeroed
        dl_g = dls[q].copy()
        dl_g[~use] = 0
        b.dl_dobs[q].copy_(torch.tensor(dl_g, dtype=torch.float32))
        b.run()
        g = b.dtheta[q].double().cpu().numpy()
        ref = orc.dtheta[use].sum(0)
        rel = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30)
        assert rel < GRAD_RTOL, (q, rel)


def test_batch_matches_oracle_on_all_256_networks(S):
    """Every network of the uneven random-network workload, four trajectories each, in one batch against
    the FP64 oracle: status codes; event sequences under the margin rule and the long-trajectory count
    rule per network, with at least 90% identical over all trajectories; observables and each network's
    gradient on the trajectories whose events and sample brackets agree."""
    from concurrent.futures import ThreadPoolExecutor
    from types import SimpleNamespace
    from oracle import native
    from test_gpu_parity import GRAD_RTOL, _bracket_agreement, _clock_tol, _compare_events, _oracle_brackets

    wl = W.config_c4(n_nets=256)
    cap = 1 << 16
    n = 4
    nets = [S.Network(spec) for spec in wl.nets]
    items = [dict(net=nets[q], log_rates=spec.log_rates.astype(np.float32), n_traj=n, x0=spec.x0,
                  t_end=wl.t_end, sample_times=wl.sample_times, obs_species=wl.obs_species[q], seed=300 + q,
                  traj_offset=7 * q, max_steps=cap) for q, spec in enumerate(wl.nets)]
    b = S.Batch(items, readout="linear", temperature=wl.temperature)
    dls = [W.seeded_dl_dobs(900 + q, n, len(wl.sample_times), len(wl.obs_species[q]), scale=1.0 / n)
           for q in range(len(items))]
    for q in range(len(items)):
        b.dl_dobs[q].copy_(torch.tensor(dls[q], dtype=torch.float32))
    b.run()
    torch.cuda.synchronize()

    def oracle(q):
        spec, it = wl.nets[q], items[q]
        return native.run(spec, spec.log_rates.astype(np.float32).astype(np.float64), spec.x0, n, wl.t_end,
                          wl.sample_times, wl.obs_species[q], it["seed"], LINEAR, max_steps=cap,
                          traj_offset=it["traj_offset"], dl_dobs=dls[q], temperature=wl.temperature, ev_cap=cap,
                          n_threads=1)

    with ThreadPoolExecutor(max_workers=16) as ex:
        orcs = list(ex.map(oracle, range(len(items))))
    uses, n_same = [], 0
    for q, spec in enumerate(wl.nets):
        orc = orcs[q]
        draws, status, mism = b.outputs(q)
        assert mism == 0
        np.testing.assert_array_equal(status.cpu().numpy(), orc.status)
        fw = SimpleNamespace(draws=draws, status=status, run=SimpleNamespace(brackets=lambda q=q: b.brackets(q)))
        same = _compare_events(orc, fw, b.events(q, cap).cpu().numpy(), wl.t_end, spec.n_reactions, floor=None)
        n_same += int(same.sum())
        use = same & _bracket_agreement(orc, fw, wl.sample_times, spec.n_reactions)
        obs = b.obs[q].double().cpu().numpy()
        ob = _oracle_brackets(orc, wl.sample_times)
        vmax = np.abs(spec.stoich_delta).max()
        for i in np.nonzero(use)[0]:
            t = np.concatenate([[0.0], orc.times[i, :orc.draws[i]]])
            k = ob[i]
            tau = t[np.minimum(k + 1, len(t) - 1)] - t[k]
            tol = vmax * _clock_tol(spec.n_reactions, wl.sample_times) / np.maximum(tau, 1e-300) \
                + 1e-6 * np.abs(orc.obs[i]).max(1)
            assert np.all(np.abs(obs[i] - orc.obs[i]).max(1) <= tol), (q, i)
        uses.append(use)
    assert n_same >= 0.9 * n * len(items), n_same
    # gradients over the agreeing trajectories of every network, from one more run of the batch
    for q in range(len(items)):
        dl_g = dls[q].copy()
        dl_g[~uses[q]] = 0
        b.dl_dobs[q].copy_(torch.tensor(dl_g, dtype=torch.float32))
    b.run()
    torch.cuda.synchronize()
    for q in range(len(items)):
        g = b.dtheta[q].double().cpu().numpy()
        ref = orcs[q].dtheta[uses[q]].sum(0)
        if not uses[q].any():
            assert np.all(g == 0)
            continue
        rel = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30)
        assert rel < GRAD_RTOL, (q, rel)


def test_batch_autotuned_checkpoint_interval_changes_no_result(S):
    """Items that leave K free get the autotuner's interval (one of the three timed multiples of 16 N); the
    results are those of the same batch with K fixed at 64 bit for bit (K only sets how often the state is
    stored and checked)."""
    wl = W.config_c4(n_nets=6, traj_scale=1.0 / 128)
    nets = [S.Network(spec) for spec in wl.nets]

    def items(K):
        return [dict(net=nets[q], log_rates=spec.log_rates.astype(np.float32), n_traj=int(wl.n_traj[q]), x0=spec.x0,
                     t_end=wl.t_end, sample_times=wl.sample_times, obs_species=wl.obs_species[q], seed=20 + q,
                     max_steps=1 << 16, **({"ckpt_interval": K} if K else {})) for q, spec in enumerate(wl.nets)]

    runs = []
    for K in (0, 64):
        b = S.Batch(items(K), readout="linear", temperature=wl.temperature)
        b.autotune(pilot_traj=16)
        for q in range(len(nets)):
            b.dl_dobs[q].copy_(torch.tensor(W.seeded_dl_dobs(q, int(wl.n_traj[q]), len(wl.sample_times),
                                                             len(wl.obs_species[q]), scale=1e-3), dtype=torch.float32))
        b.run()
        torch.cuda.synchronize()
        runs.append(b)
    free, fixed = runs
    for q, spec in enumerate(wl.nets):
        base = min(1024, max(16, (16 * spec.n_species + 7) // 8 * 8))
        assert free.ckpt_interval(q) in {min(4096, max(8, int(c * base / 8.0 + 0.5) * 8)) for c in (0.25, 1.0, 4.0)}
        assert fixed.ckpt_interval(q) == 64
        assert torch.equal(free.obs[q], fixed.obs[q]) and torch.equal(free.dtheta[q], fixed.dtheta[q]), q
        assert free.outputs(q)[2] == 0 and fixed.outputs(q)[2] == 0


@pytest.mark.parametrize("shared", [False, True])
def test_batch_bin_readout_matches_single_network_entry_points(S, specs, shared):
    """The bin readout (Section 4.4) in the batch: thread units and warp units give the bin averages of the
    single-network calls bit for bit and their gradients to binary32 rounding, with one upstream gradient
    per trajectory or one shared by all of an item's trajectories (the binary64 prefix sums)."""
    nets = [S.Network(sp[0]) for sp in specs]
    items = _items(S, specs, nets)
    for it in items:
        it["obs_species"] = it["obs_species"][:4]
        it["shared_dl"] = shared
    b = S.Batch(items, readout="bin", temperature=0.6)
    for q, (net, n, t_end, ns, obs, *_rest) in enumerate(specs):
        shape = (1, ns, len(items[q]["obs_species"])) if shared else (n, ns, len(items[q]["obs_species"]))
        dl = W.seeded_dl_dobs(40 + q, *shape, scale=1.0 / max(n, 1))
        b.dl_dobs[q].copy_(torch.tensor(dl[0] if shared else dl, dtype=torch.float32))
    b.run()
    torch.cuda.synchronize()
    _check_against_single(S, b, specs, nets, items, 0.6, readout="bin")


def test_soft_batch_matches_single_network_warp_calls(S, specs):
    """ssa_batch_set_soft: every item runs the soft forward (Eq. 4) and the exact gradient of the relaxed model
    as warp units; observables, draws and status equal the single-network warp soft calls bit for bit (the same
    per-trajectory bodies), gradients to binary32 summation order. T = 2, where these relaxed models are well
    conditioned."""
    T = 2.0
    sp = [specs[0], specs[1], specs[3], specs[5], specs[6]]
    nets = [S.Network(s[0]) for s in sp]
    items = _items(S, sp, nets)
    for it in items:
        it["threads_per_traj"] = 0
    b = S.Batch(items, readout="linear", temperature=T, soft=True)
    assert all(b.variant(q) == 32 for q in range(len(sp)))
    _fill_dl(b, sp)
    b.run()
    for q in range(len(sp)):
        it = items[q]
        fw = S.forward(nets[q], torch.tensor(it["log_rates"], device="cuda"), it["n_traj"], it["x0"], it["t_end"],
                       it["sample_times"], it["obs_species"], it["seed"], readout="linear", record=True,
                       max_steps=it["max_steps"], traj_offset=it["traj_offset"], threads_per_traj=32,
                       selector="soft", temperature=T)
        draws, status, mism = b.outputs(q)
        assert mism == 0
        assert torch.equal(b.obs[q], fw.obs), q
        assert torch.equal(draws, fw.draws) and torch.equal(status, fw.status), q
        if it["n_traj"] == 0:
            assert torch.all(b.dtheta[q] == 0)
            continue
        g = S.backward(fw, b.dl_dobs[q], T).double().cpu().numpy()
        gb = b.dtheta[q].double().cpu().numpy()
        scale = max(np.abs(g).max(), 1e-12)
        assert np.abs(gb - g).max() <= 1e-4 * scale, (q, np.abs(gb - g).max(), scale)
    # no event log in a soft batch; threads are refused
    from paper_2602_19775_gb300 import SSAError
    with pytest.raises(SSAError):
        b.events(0, 64)
    with pytest.raises(SSAError):
        b.set_plan(0, 1, 64)
