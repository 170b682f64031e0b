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


# ---------------------------------------------------------------------------------------------
# The soft forward of Eq. 4 on the GRN (the first training phase of Section 3.5)
# ---------------------------------------------------------------------------------------------
def test_soft_grn_at_low_temperature_is_the_hard_path():
    """T -> 0: the soft sample is one-hot on the Gumbel-max choice; where every key gap exceeds 1e-4,
    T = 1e-9 leaves exp(-1e5) on the other reactions and the soft path is the hard one exactly."""
    p, x = _tiny()
    ts = np.array([1.0, 3.0, 6.0])
    hard = native.grn_run(p, x, 16, 6.0, ts, 3, ev_cap=4000)
    soft = native.grn_run(p, x, 16, 6.0, ts, 3, ev_cap=4000, soft=True, temperature=1e-9)
    clear = np.array([np.nanmin(hard.margins[i, :hard.draws[i]]) > 1e-4 for i in range(32)])
    assert clear.sum() >= 8
    np.testing.assert_array_equal(soft.obs[clear], hard.obs[clear])
    np.testing.assert_array_equal(soft.events[clear], hard.events[clear])


def _soft_refs(r, i, x):
    return {"W1": np.outer(r.dE1[i], x), "b1": r.dE1[i], "W2": r.dW2[i], "b2": r.db2[i], "log_d": r.dlogd[i]}


def test_soft_grn_hand_adjoint_matches_autograd():
    """The exact gradient of the relaxed GRN (hand adjoint along the soft path) against float64 autograd of
    the relaxed graph at two temperatures; relaxed counts go below 0 at both (about 6% of the output samples at
    T = 0.6), so the clipped degradation (a zero propensity, masked from the soft sample) is exercised. With
    the HOLD readout the waiting time carries no gradient, so the clip's own derivative never enters."""
    p, x = _tiny()
    ts = np.array([1.0, 3.0, 6.0])
    for T in (0.6, 3.0):
        dl = np.random.default_rng(5).standard_normal((4, 3, 3))
        r = native.grn_run(p, x, 2, 6.0, ts, 9, dl_dobs=dl, temperature=T, ev_cap=4000, soft=True)
        assert np.all(r.status == 0)
        for i in range(4):
            nd = int(r.draws[i])
            g = autodiff.grn_st_gradient(p, x[i // 2], r.events[i, :nd], nd, True, 9, i, ts, dl[i], T, soft=True)
            ref = _soft_refs(r, i, x[i // 2])
            for k in g:
                scale = max(np.abs(g[k]).max(), 1e-300)
                assert np.abs(g[k] - ref[k]).max() / scale < 1e-9, (T, i, k)


def test_soft_grn_gradient_matches_finite_differences():
    """For fixed noise the soft path is smooth in the parameters (while its step count does not change),
    so the relaxed model's gradient is the limit of central differences."""
    import dataclasses
    p, x = _tiny()
    p = dataclasses.replace(p, W1=p.W1.astype(np.float64), b1=p.b1.astype(np.float64), W2=p.W2.astype(np.float64),
                            b2=p.b2.astype(np.float64), log_d=p.log_d.astype(np.float64))
    ts = np.array([1.0, 3.0, 6.0])
    T, h = 0.8, 1e-6
    dl = np.random.default_rng(6).standard_normal((4, 3, 3))
    base = native.grn_run(p, x, 2, 6.0, ts, 13, dl_dobs=dl, temperature=T, soft=True)
    for name, idx in (("b2", (1,)), ("W2", (0, 2)), ("log_d", (5,)), ("b1", (2,)), ("W1", (1, 4))):
        arr = getattr(p, name)
        plus, minus = arr.copy(), arr.copy()
        plus[idx] += h
        minus[idx] -= h
        rp = native.grn_run(dataclasses.replace(p, **{name: plus}), x, 2, 6.0, ts, 13, temperature=T, soft=True)
        rm = native.grn_run(dataclasses.replace(p, **{name: minus}), x, 2, 6.0, ts, 13, temperature=T, soft=True)
        same = (rp.draws == base.draws) & (rm.draws == base.draws)
        assert same.sum() >= 3
        fd = ((rp.obs - rm.obs) * dl).sum((1, 2)) / (2 * h)
        for i in np.nonzero(same)[0]:
            g = _soft_refs(base, i, x[i // 2])[name][idx]
            assert abs(fd[i] - g) <= 1e-5 * max(abs(g), 1e-3), (name, i, fd[i], g)
