"""GPU parity of the gene-regulatory-network classifier (Section 4.3) against the FP64 oracle:
the tensor-core activation energies E1 = W1 x + b1 (exact up to one rounding), the event
sequences (margin rule), the HOLD observables, and every gradient group on the trajectories whose
events agree."""
import numpy as np
import pytest
import torch

from ssa_workloads import grn as G
from oracle import native

from test_gpu_parity import GRAD_RTOL, _divergence_rule

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2602_19775_gb300 import ssa
    ssa._lib.lib()
    return ssa


@pytest.mark.parametrize("n_img", [512, 40, 5000])
def test_activation_energies_are_exact_on_tensor_cores(S, n_img):
    """512 images: 16 output tiles, K split 7 ways (int64 limb pairs added across the splits); 40: one tile row;
    5,000: 160 tiles, no split (the limb sum in the GEMM's own epilogue)."""
    p = G.grn_params(seed=5)
    p.b1[:] = np.random.default_rng(1).normal(0, 0.5, p.n_hid).astype(np.float32)
    x, _ = G.prototype_images(seed=5, n_img=n_img)
    net = S.GRN(p.n_in, p.n_hid, p.n_out, p.k_max)
    fw = S.grn_forward(net, p.W1, p.b1, p.W2, p.b2, p.log_d, x, 1, 0.0, [0.0], 3, record=False)
    E1, flags = S.grn_activations(fw, n_img)
    assert flags == (0, 0), flags
    # W1 x is exact in binary64 (bf16 weights times 8-bit counts on one grid); one rounding of (W1 x + b1)
    exact = x.astype(np.float64) @ p.W1.astype(np.float64).T + p.b1.astype(np.float64)
    np.testing.assert_array_equal(E1.cpu().numpy(), exact.astype(np.float32))


def _grn_case(S, p, x, tpi, t_end, seed, T, max_steps=1 << 15):
    n = x.shape[0] * tpi
    ts = np.array([t_end])
    dl = np.random.default_rng(seed + 1).standard_normal((n, 1, p.n_out)) / n
    net = S.GRN(p.n_in, p.n_hid, p.n_out, p.k_max)
    fw = S.grn_forward(net, p.W1, p.b1, p.W2, p.b2, p.log_d, x, tpi, t_end, ts, seed, max_steps=max_steps)
    orc = native.grn_run(p, x, tpi, t_end, ts, seed, max_steps=max_steps, dl_dobs=dl, temperature=T, ev_cap=max_steps)
    assert np.all(fw.status.cpu().numpy() == orc.status)
    ev = fw.run.events(max_steps).cpu().numpy()
    # margin rule at each first divergence and the long-trajectory count rule (532 reactions per race,
    # thousands of draws), beside a floor of 0.95
    same = _divergence_rule(ev, fw.draws.cpu().numpy(), orc)
    assert same.mean() >= 0.95, same.mean()
    obs = fw.obs.double().cpu().numpy()
    np.testing.assert_array_equal(obs[same], orc.obs[same])
    dl_g = dl.copy()
    dl_g[~same] = 0
    g = S.grn_backward(fw, torch.tensor(dl_g, dtype=torch.float32, device="cuda"), T)
    keep = np.repeat(same, 1)
    masked = native.GRNResult(orc.obs, orc.draws, orc.status, orc.dE1 * keep[:, None], orc.dW2 * keep[:, None, None],
                              orc.db2 * keep[:, None], orc.dlogd * keep[:, None], None, None)
    ref = masked.grads(x, tpi)
    _, mism = fw.run.status_counts()
    assert mism == 0
    errs = {}
    for k in ref:
        gk = g[k].double().cpu().numpy()
        errs[k] = np.linalg.norm(gk - ref[k]) / max(np.linalg.norm(ref[k]), 1e-300)
    assert all(e < GRAD_RTOL for e in errs.values()), errs
    return errs, same.mean()


def test_tiny_grn_matches_oracle(S):
    p = G.grn_params(seed=1, n_in=5, n_hid=4, n_out=3, w1_scale=0.02, w2_scale=0.5)
    p.b1[:] = [0.3, -0.5, 1.0, 0.0]
    p.b2[:] = [0.2, -0.1, 0.4]
    x = np.array([[10, 200, 3, 0, 77], [5, 5, 5, 250, 1], [0, 0, 0, 0, 0]], np.int32)
    _grn_case(S, p, x, 256, 6.0, 7, 0.6)


def test_mnist_sized_grn_matches_oracle(S):
    p = G.grn_params(seed=5)
    x, _ = G.prototype_images(seed=5, n_img=4)
    _grn_case(S, p, x, 8, 4.0, 9, 1.0)


@pytest.mark.parametrize("size", ["tiny", "mnist_shape"])
def test_grn_soft_forward_matches_oracle(S, size):
    """The soft forward of Eq. 4 on the GRN (the first training phase of Section 3.5) against the oracle's on
    the same noise. The relaxed path is smooth in its noise, so the binary32 GPU path drifts from the binary64
    one by roundoff amplified by the dynamics: the bound per sample is k 64 2^-24 (max|X| + 1) after k steps
    plus 4 x the oracle's response to a perturbation of the biases and degradation rates scaled to 64 ulp;
    required on 99% of the samples and for every sample's ensemble mean."""
    import dataclasses
    if size == "tiny":
        p = G.grn_params(seed=1, n_in=5, n_hid=4, n_out=3, w1_scale=0.02, w2_scale=0.5)
        p.b1[:] = [0.3, -0.5, 1.0, 0.0]
        p.b2[:] = [0.2, -0.1, 0.4]
        x = np.array([[10, 200, 3, 0, 77], [5, 5, 5, 250, 1]], np.int32)
        tpi, t_end, T = 64, 6.0, 0.7
    else:
        p = G.grn_params(seed=5)
        x, _ = G.prototype_images(seed=5, n_img=4)
        tpi, t_end, T = 16, 4.0, 1.0
    ts = np.linspace(t_end / 8, t_end, 8)
    net = S.GRN(p.n_in, p.n_hid, p.n_out, p.k_max)
    fw = S.grn_forward(net, p.W1, p.b1, p.W2, p.b2, p.log_d, x, tpi, t_end, ts, 3, soft_temperature=T,
                       max_steps=1 << 14)
    T32 = float(np.float32(T))
    pd = dataclasses.replace(p, W1=p.W1.astype(np.float64), b1=p.b1.astype(np.float64), W2=p.W2.astype(np.float64),
                             b2=p.b2.astype(np.float64), log_d=p.log_d.astype(np.float64))
    orc = native.grn_run(pd, x, tpi, t_end, ts, 3, max_steps=1 << 14, soft=True, temperature=T32, ev_cap=1 << 14)
    st = fw.status.cpu().numpy()
    assert np.all(st == orc.status)
    same = fw.draws.cpu().numpy() == orc.draws
    assert same.mean() > 0.95
    delta = 1e-6
    sens = np.zeros_like(orc.obs)
    for name in ("b1", "b2", "log_d"):
        o2 = native.grn_run(dataclasses.replace(pd, **{name: getattr(pd, name) + delta}), x, tpi, t_end, ts, 3,
                            max_steps=1 << 14, soft=True, temperature=T32)
        sens += np.abs(o2.obs - orc.obs)
    amp = 4 * 64 * 2.0 ** -24 / delta * sens
    obs = fw.obs.double().cpu().numpy()
    idx = np.nonzero(same)[0]
    k = orc.draws[idx].astype(float)[:, None, None]
    xmax = np.abs(orc.obs[idx]).max(axis=(1, 2), keepdims=True) + 1.0
    bound = (k + 1) * 64 * 2.0 ** -24 * xmax + amp[idx]
    err = np.abs(obs[idx] - orc.obs[idx])
    assert (err <= bound).mean() >= 0.99, ((err <= bound).mean(), err.max())
    assert np.all(np.abs((obs[idx] - orc.obs[idx]).mean(0)) <= bound.mean(0))


@pytest.mark.parametrize("size", ["tiny", "mnist_shape"])
def test_grn_soft_gradient_matches_oracle(S, size):
    """The exact gradient of the relaxed GRN (the soft forward of Eq. 4, differentiated along its own path) against
    the oracle's on the same noise. One sample at t_end reads the last state, so a trajectory with the oracle's
    draw count has the oracle's bracket; the others (a crossing decided within the clock tolerance) are left out.
    The path is smooth in its parameters, so binary32 against binary64 differ by roundoff: over the 1e2 steps of
    these runs about 1e2 x 64 ulp per trajectory at worst, averaging down over the ensemble: 2e-3 in norm."""
    import dataclasses
    if size == "tiny":
        p = G.grn_params(seed=1, n_in=5, n_hid=4, n_out=3, w1_scale=0.02, w2_scale=0.5)
        p.b1[:] = [0.3, -0.5, 1.0, 0.0]
        p.b2[:] = [0.2, -0.1, 0.4]
        x = np.array([[10, 200, 3, 0, 77], [5, 5, 5, 250, 1]], np.int32)
        tpi, t_end, T = 128, 6.0, 0.7
    else:
        p = G.grn_params(seed=5)
        x, _ = G.prototype_images(seed=5, n_img=4)
        tpi, t_end, T = 16, 1.0, 1.0
    n = x.shape[0] * tpi
    ts = np.array([t_end])
    T32 = float(np.float32(T))
    dl = np.random.default_rng(21).standard_normal((n, 1, p.n_out)) / n
    net = S.GRN(p.n_in, p.n_hid, p.n_out, p.k_max)
    fw = S.grn_forward(net, p.W1, p.b1, p.W2, p.b2, p.log_d, x, tpi, t_end, ts, 13, soft_temperature=T,
                       max_steps=1 << 12)
    pd = dataclasses.replace(p, W1=p.W1.astype(np.float64), b1=p.b1.astype(np.float64), W2=p.W2.astype(np.float64),
                             b2=p.b2.astype(np.float64), log_d=p.log_d.astype(np.float64))
    orc = native.grn_run(pd, x, tpi, t_end, ts, 13, max_steps=1 << 12, soft=True, temperature=T32, dl_dobs=dl,
                         ev_cap=1 << 12)
    assert np.all(fw.status.cpu().numpy() == orc.status)
    same = fw.draws.cpu().numpy() == orc.draws
    assert same.mean() > 0.95
    dl_g = dl.copy()
    dl_g[~same] = 0
    g = S.grn_backward(fw, torch.tensor(dl_g, dtype=torch.float32, device="cuda"), T)
    _, mism = fw.run.status_counts()
    assert mism == 0  # every re-run segment ends on its checkpoint, bit for bit
    masked = native.GRNResult(orc.obs, orc.draws, orc.status, orc.dE1 * same[:, None], orc.dW2 * same[:, None, None],
                              orc.db2 * same[:, None], orc.dlogd * same[:, None], None, None)
    ref = masked.grads(x, tpi)
    errs = {k: np.linalg.norm(g[k].double().cpu().numpy() - ref[k]) / max(np.linalg.norm(ref[k]), 1e-300)
            for k in ref}
    assert all(e < 2e-3 for e in errs.values()), errs
    # the observables of a recorded soft run are those of an unrecorded one
    fw2 = S.grn_forward(net, p.W1, p.b1, p.W2, p.b2, p.log_d, x, tpi, t_end, ts, 13, soft_temperature=T,
                        max_steps=1 << 12, record=False)
    assert torch.equal(fw.obs, fw2.obs)
    with pytest.raises(RuntimeError):  # the relaxed model's gradient is at its own temperature
        S.grn_backward(fw, torch.tensor(dl_g, dtype=torch.float32, device="cuda"), 2 * T)
    with pytest.raises(RuntimeError):  # a soft run keeps no event log
        fw.run.events(16)


@pytest.mark.parametrize("soft", [False, True], ids=["hard", "soft"])
def test_grn_empty_batch(S, soft):
    """No images: the forward writes nothing and the backward returns zero gradients."""
    p = G.grn_params(seed=1, n_in=5, n_hid=4, n_out=3, w1_scale=0.02, w2_scale=0.5)
    net = S.GRN(p.n_in, p.n_hid, p.n_out, p.k_max)
    x = np.zeros((0, 5), np.int32)
    fw = S.grn_forward(net, p.W1, p.b1, p.W2, p.b2, p.log_d, x, 8, 2.0, [1.0, 2.0], 3,
                       soft_temperature=0.5 if soft else None)
    assert fw.obs.shape == (0, 2, 3) and fw.draws.numel() == 0
    g = S.grn_backward(fw, torch.zeros((0, 2, 3), device="cuda"), 0.5)
    for k, v in g.items():
        assert torch.count_nonzero(v) == 0, k
