"""The seeded input generators (`ssa_workloads`), which both the oracle and the GPU path take their inputs
from: deterministic under a seed, and of the shapes, ranges and structure their docstrings state."""
import numpy as np

import ssa_workloads as W
from ssa_workloads import grn as G
from ssa_workloads.networks import random_network


def test_sample_grid_ends_exactly_at_the_horizon():
    for t_end, S in ((50.0, 50), (0.05, 3), (400.0, 400), (1.0 / 3.0, 7)):
        ts = W.uniform_sample_grid(t_end, S)
        assert ts.shape == (S,) and ts[-1] == t_end and np.all(np.diff(ts) > 0) and ts[0] > 0


def test_reference_workloads():
    c2 = W.config_c2()
    assert c2.n_traj == 65536 and c2.t_end == 50.0 and len(c2.sample_times) == 50 and c2.readout == W.configs.LINEAR
    assert np.allclose(np.exp(c2.log_rates), [0.02, 0.05]) and c2.temperatures == (0.1, 0.5, 1.0)
    V = c2.net.stoich_dense()
    assert np.array_equal(V @ np.array([1, 2]), np.zeros(V.shape[0]))  # A + 2B is conserved
    c3 = W.config_c3(n_traj=8)
    assert c3.net.n_species == 9 and c3.net.n_reactions == 16 and len(c3.sample_times) == 400


def test_seeded_generators_are_deterministic():
    a = W.seeded_dl_dobs(3, 16, 5, 2)
    assert np.array_equal(a, W.seeded_dl_dobs(3, 16, 5, 2)) and not np.array_equal(a, W.seeded_dl_dobs(4, 16, 5, 2))
    p1, p2 = G.grn_params(seed=7, n_in=20, n_hid=8, n_out=3), G.grn_params(seed=7, n_in=20, n_hid=8, n_out=3)
    assert np.array_equal(p1.W1, p2.W1) and np.array_equal(p1.W2, p2.W2)
    x1, l1 = G.prototype_images(seed=2, n_img=30, n_in=20)
    x2, l2 = G.prototype_images(seed=2, n_img=30, n_in=20)
    assert np.array_equal(x1, x2) and np.array_equal(l1, l2)
    n1 = random_network(np.random.default_rng(9))
    n2 = random_network(np.random.default_rng(9))
    assert np.array_equal(n1.reactants, n2.reactants) and np.array_equal(n1.log_rates, n2.log_rates)


def test_grn_inputs():
    p = G.grn_params()
    assert p.W1.shape == (256, 784) and p.W2.shape == (10, 256) and p.log_d.shape == (266,)
    # bf16-representable: the low 16 bits of every binary32 weight are zero
    assert np.all(p.W1.view(np.uint32) & 0xFFFF == 0) and np.all(p.W2.view(np.uint32) & 0xFFFF == 0)
    x, labels = G.prototype_images(n_img=100)
    assert x.dtype == np.int32 and x.min() >= 0 and x.max() <= 255 and x.shape == (100, 784)
    assert np.array_equal(labels, np.arange(100) % 10)


def test_round_bf16_is_nearest_even():
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)  # bf16 spacing at 1
    vals = np.array([one + ulp / 2, one + 3 * ulp / 2, one + ulp / 4, -(one + 3 * ulp / 4)], np.float32)
    np.testing.assert_array_equal(G.round_bf16(vals), np.array([one, one + 2 * ulp, one, -(one + ulp)], np.float32))


def test_random_networks_keep_counts_non_negative_by_construction():
    rng = np.random.default_rng(11)
    for _ in range(20):
        net = random_network(rng, n_species_range=(2, 12), n_reactions_range=(4, 40))
        V = net.stoich_dense()
        assert 2 <= net.n_species <= 12 and 4 <= net.n_reactions <= 40
        assert np.abs(V).max() <= 2
        for j in range(net.n_reactions):
            need = np.zeros(net.n_species, int)
            for r in net.reactants[j]:
                if r >= 0:
                    need[r] += 1
            # a reaction consumes at most what its own reactants hold when it fires
            assert np.all(-V[j] <= need), (j, V[j], need)
