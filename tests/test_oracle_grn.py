"""Pins of the GRN oracle (Section 4.3): the hand adjoint against float64 autograd of the literal
straight-through graph, and the forward law against the Poisson law of immigration-death, which is
what each gene reduces to when no gene regulates another (W2 = 0)."""
import numpy as np

from ssa_workloads import grn as G
from oracle import autodiff, cme, native


def _tiny():
    p = G.grn_params(seed=1, n_in=5, n_hid=4, n_out=3, w1_scale=0.02, w2_scale=0.5)
    p.b1[:] = [0.3, -0.5, 1.0, 0.0]
    p.b2[:] = [0.2, -0.1, 0.4]
    p.log_d[:] = np.log([0.5, 0.3, 0.8, 0.4, 0.6, 0.25, 0.9]).astype(np.float32)
    x = np.array([[10, 200, 3, 0, 77], [5, 5, 5, 250, 1]], np.int32)
    return p, x


def test_bf16_rounding_of_weights():
    p = G.grn_params(seed=3, n_in=784, n_hid=256, n_out=10)
    for W in (p.W1, p.W2):
        bits = W.view(np.uint32)
        assert np.all(bits & 0xFFFF == 0)  # representable in bfloat16


def test_grn_hand_adjoint_matches_autograd():
    p, x = _tiny()
    ts = np.array([1.0, 3.0, 6.0])
    dl = np.random.default_rng(2).standard_normal((4, 3, 3))
    r = native.grn_run(p, x, 2, 6.0, ts, 7, dl_dobs=dl, temperature=0.6, ev_cap=4000)
    assert np.all(r.status == 0)
    for i in range(4):
        nd = int(r.draws[i])
        g = autodiff.grn_st_gradient(p, x[i // 2], r.events[i, :nd], nd, True, 7, i, ts, dl[i], 0.6)
        ref = {"W1": np.outer(r.dE1[i], x[i // 2]), "b1": r.dE1[i], "W2": r.dW2[i], "b2": r.db2[i],
               "log_d": r.dlogd[i]}
        for k in g:
            scale = max(np.abs(g[k]).max(), 1e-300)
            assert np.abs(g[k] - ref[k]).max() / scale < 1e-10, (i, k)


def test_grn_without_regulation_is_immigration_death():
    p = G.grn_params(seed=2, n_in=3, n_hid=1, n_out=1, w1_scale=0.01)
    p.W2[:] = 0.0
    p.b1[:] = 0.4
    p.b2[:] = -0.7
    p.log_d[:] = np.log([0.5, 0.8]).astype(np.float32)
    p.k_max = 3.0
    x = np.array([[100, 20, 5]], np.int32)
    n = 20000
    ts = np.array([0.5, 2.0, 8.0])
    r = native.grn_run(p, x, n, 8.0, ts, 11)
    y = r.obs[:, :, 0]
    lam = p.k_max / (1.0 + np.exp(-float(p.b2[0])))
    mean = cme.immigration_death_mean(lam, 0.8, ts)
    se = np.sqrt(mean / n)
    assert np.all(np.abs(y.mean(0) - mean) < 3 * se), (y.mean(0), mean)
