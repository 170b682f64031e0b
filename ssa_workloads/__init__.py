"""Seeded synthetic inputs shared by the tests, the benchmark and both implementations.

This package holds reaction-network descriptions, sample grids, initial states and seeded random
draws (loss weights, random networks, synthetic images). It holds none of the simulation or
gradient arithmetic: the CPU oracle and the CUDA library each implement that on their own and
both take these inputs as plain integer/float arrays.
"""
from .networks import (  # noqa: F401
    NetworkSpec,
    network_from_reactions,
    dimerization_2a_b,
    dimerization_a_b_c,
    immigration_death,
    vilar_oscillator,
    ion_channel_coi,
    mixed_orders_toy,
    random_network,
)
from .configs import (  # noqa: F401
    uniform_sample_grid,
    config_c1,
    config_c2,
    config_c3,
    config_c4,
    seeded_dl_dobs,
)
