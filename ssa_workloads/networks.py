"""Reaction networks as plain arrays.

A network is a list of reactions; each reaction names up to two reactant species (mass-action
order 0, 1 or 2, a repeated species meaning a homodimer), its product species, and the name of
the log-rate parameter it uses. ``network_from_reactions`` turns that list into the array form
both implementations read:

* ``reactants``   int32 [M, 2]   reactant species per reaction, -1 for an empty slot
* ``stoich_ptr``  int32 [M + 1]  CSR row pointer of the net change v_j
* ``stoich_species`` / ``stoich_delta`` int32 [nnz]  non-zero entries of v_j (species, change)
* ``rate_index``  int32 [M]      which parameter of ``log_rates`` reaction j uses

Network models follow arXiv 2602.19775: the reversible dimerization of Section 4.1 (Eq. 8), the
activator-repressor oscillator of Section 4.2 (the model of its reference 30), the C/O/I channel
of Section 4.4, and a 2A <-> B variant with a homodimer propensity k A (A - 1) / 2 (Section 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Sequence

import numpy as np


@dataclass(frozen=True)
class NetworkSpec:
    species: tuple
    reactants: np.ndarray
    stoich_ptr: np.ndarray
    stoich_species: np.ndarray
    stoich_delta: np.ndarray
    param_names: tuple
    rate_index: np.ndarray
    log_rates: np.ndarray = field(default=None)  # default parameter point (float64), may be None
    x0: np.ndarray = field(default=None)         # default initial state (int32), may be None

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return int(self.reactants.shape[0])

    @property
    def n_params(self) -> int:
        return len(self.param_names)

    def species_index(self, name: str) -> int:
        return self.species.index(name)

    def stoich_dense(self) -> np.ndarray:
        """[M, N] net change matrix (a convenience view of the CSR arrays)."""
        V = np.zeros((self.n_reactions, self.n_species), dtype=np.int64)
        for j in range(self.n_reactions):
            for e in range(self.stoich_ptr[j], self.stoich_ptr[j + 1]):
                V[j, self.stoich_species[e]] += self.stoich_delta[e]
        return V


def network_from_reactions(species: Sequence[str], reactions, rates: dict | None = None,
                           x0: dict | None = None) -> NetworkSpec:
    """reactions: iterable of (reactants, products, param_name) with species names."""
    species = tuple(species)
    sidx = {s: i for i, s in enumerate(species)}
    params: list[str] = []
    react, ptr, sp, dl, ridx = [], [0], [], [], []
    for reac, prod, pname in reactions:
        reac = list(reac)
        if len(reac) > 2:
            raise ValueError("mass-action order above 2 is not supported")
        slots = [sidx[r] for r in reac] + [-1] * (2 - len(reac))
        react.append(slots)
        net: dict[int, int] = {}
        for r in reac:
            net[sidx[r]] = net.get(sidx[r], 0) - 1
        for p in prod:
            net[sidx[p]] = net.get(sidx[p], 0) + 1
        for s_i in sorted(net):
            if net[s_i] != 0:
                sp.append(s_i)
                dl.append(net[s_i])
        ptr.append(len(sp))
        if pname not in params:
            params.append(pname)
        ridx.append(params.index(pname))
    log_rates = None
    if rates is not None:
        log_rates = np.log(np.array([float(rates[p]) for p in params], dtype=np.float64))
    x0_arr = None
    if x0 is not None:
        x0_arr = np.array([int(x0.get(s, 0)) for s in species], dtype=np.int32)
    return NetworkSpec(
        species=species,
        reactants=np.array(react, dtype=np.int32).reshape(-1, 2),
        stoich_ptr=np.array(ptr, dtype=np.int32),
        stoich_species=np.array(sp, dtype=np.int32),
        stoich_delta=np.array(dl, dtype=np.int32),
        param_names=tuple(params),
        rate_index=np.array(ridx, dtype=np.int32),
        log_rates=log_rates,
        x0=x0_arr,
    )


def dimerization_2a_b(k1: float = 0.01, k2: float = 0.1, a0: int = 100) -> NetworkSpec:
    """2A <-> B with a1 = k1 A (A - 1) / 2 and a2 = k2 B; A + 2B is conserved."""
    return network_from_reactions(
        ["A", "B"],
        [(["A", "A"], ["B"], "k1"), (["B"], ["A", "A"], "k2")],
        rates={"k1": k1, "k2": k2}, x0={"A": a0, "B": 0})


def dimerization_a_b_c(k1: float = 0.01, k2: float = 0.32, xa: int = 100, xb: int = 90) -> NetworkSpec:
    """A + B <-> C (Eq. 8): a1 = k1 A B, a2 = k2 C."""
    return network_from_reactions(
        ["A", "B", "C"],
        [(["A", "B"], ["C"], "k1"), (["C"], ["A", "B"], "k2")],
        rates={"k1": k1, "k2": k2}, x0={"A": xa, "B": xb, "C": 0})


def immigration_death(lam: float = 10.0, mu: float = 1.0) -> NetworkSpec:
    """0 -> A at rate lam, A -> 0 at rate mu A."""
    return network_from_reactions(
        ["A"], [([], ["A"], "lam"), (["A"], [], "mu")],
        rates={"lam": lam, "mu": mu}, x0={"A": 0})


# Rates of the activator-repressor oscillator as listed for the oscillator workload.
VILAR_RATES = dict(alphaA=50.0, alphaA_p=500.0, alphaR=0.01, alphaR_p=50.0, betaA=50.0, betaR=5.0,
                   deltaMA=10.0, deltaMR=0.5, deltaA=1.0, deltaR=0.2, gammaA=1.0, gammaR=1.0,
                   gammaC=2.0, thetaA=50.0, thetaR=100.0)


def vilar_oscillator(rates: dict | None = None) -> NetworkSpec:
    """Activator-repressor oscillator: 9 species, 16 reactions, 15 rates (deltaA is shared by
    A -> 0 and by C -> R, the repressor released when the complexed activator decays)."""
    r = dict(VILAR_RATES)
    if rates:
        r.update(rates)
    species = ["DA", "DA_p", "DR", "DR_p", "MA", "MR", "A", "R", "C"]
    reactions = [
        (["DA", "A"], ["DA_p"], "gammaA"),
        (["DA_p"], ["DA", "A"], "thetaA"),
        (["DR", "A"], ["DR_p"], "gammaR"),
        (["DR_p"], ["DR", "A"], "thetaR"),
        (["DA_p"], ["DA_p", "MA"], "alphaA_p"),
        (["DA"], ["DA", "MA"], "alphaA"),
        (["DR_p"], ["DR_p", "MR"], "alphaR_p"),
        (["DR"], ["DR", "MR"], "alphaR"),
        (["MA"], ["MA", "A"], "betaA"),
        (["MR"], ["MR", "R"], "betaR"),
        (["A", "R"], ["C"], "gammaC"),
        (["C"], ["R"], "deltaA"),
        (["A"], [], "deltaA"),
        (["R"], [], "deltaR"),
        (["MA"], [], "deltaMA"),
        (["MR"], [], "deltaMR"),
    ]
    return network_from_reactions(species, reactions, rates=r, x0={"DA": 1, "DR": 1})


def ion_channel_coi(k_open: float = 0.75, k_close: float = 0.1, k_inact: float = 1.2,
                    n_channels: int = 2) -> NetworkSpec:
    """Three-state channel C <-> O -> I with first-order transitions (Section 4.4)."""
    return network_from_reactions(
        ["C", "O", "I"],
        [(["C"], ["O"], "k_open"), (["O"], ["C"], "k_close"), (["O"], ["I"], "k_inact")],
        rates={"k_open": k_open, "k_close": k_close, "k_inact": k_inact}, x0={"C": n_channels})


def mixed_orders_toy() -> NetworkSpec:
    """A small network with every mass-action form (orders 0, 1, hetero 2, homodimer 2) and a
    rate shared by two reactions; used for gradient cross-checks."""
    return network_from_reactions(
        ["A", "B", "C"],
        [([], ["A"], "kin"),
         (["A", "A"], ["B"], "kdim"),
         (["B"], ["A", "A"], "kun"),
         (["A", "B"], ["C"], "kab"),
         (["C"], ["A"], "kc"),
         (["B"], [], "kdeg"),
         (["C"], [], "kdeg")],
        rates={"kin": 2.0, "kdim": 0.05, "kun": 0.5, "kab": 0.02, "kc": 0.3, "kdeg": 0.1},
        x0={"A": 6, "B": 1, "C": 0})


def random_network(rng: np.random.Generator, n_species_range=(2, 64), n_reactions_range=(4, 512),
                   log10_rate_range=(-3.0, 1.0), x0_mean: float = 50.0) -> NetworkSpec:
    """A random mass-action network of the uneven-batch workload.

    Species count and reaction count are uniform in the given ranges; each reaction has two
    reactant slots, each empty or a uniformly chosen species (order 0, 1 or 2); products are
    chosen so that every net change lies in {-2..2} and a reaction only consumes its own
    reactants, so counts stay non-negative under mass action. Every reaction has its own rate,
    log10 k ~ U[range]; initial counts ~ Poisson(x0_mean).
    """
    N = int(rng.integers(n_species_range[0], n_species_range[1] + 1))
    M = int(rng.integers(n_reactions_range[0], n_reactions_range[1] + 1))
    names = [f"S{i}" for i in range(N)]
    reactions = []
    rates = {}
    for j in range(M):
        order = int(rng.integers(0, 3))
        reac = [names[int(rng.integers(0, N))] for _ in range(order)]
        n_prod = int(rng.integers(0, 3))
        prod = [names[int(rng.integers(0, N))] for _ in range(n_prod)]
        pname = f"k{j}"
        reactions.append((reac, prod, pname))
        rates[pname] = 10.0 ** rng.uniform(*log10_rate_range)
    x0 = {s: int(v) for s, v in zip(names, rng.poisson(x0_mean, size=N))}
    return network_from_reactions(names, reactions, rates=rates, x0=x0)
