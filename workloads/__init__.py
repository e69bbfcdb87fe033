"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA-side tests.

This module only *describes* reaction networks and run settings (species
count, reactant / product matrices, rate constants, initial state, grid size,
trajectory count, seed).  It contains none of the simulation arithmetic: no
propensity, no random-number mapping, no time step, no reduction.  Both the
oracle (``oracle/``) and the CUDA library (``paper_1007_1768_gb300``) take the
arrays it returns as plain inputs.

The networks follow the paper's model format (Sec. 3.2, "The StochKit-FF
implementation of the HIV model"): an integer state vector, an integer
stoichiometric description and mass-action propensities.  Reactions are given
as a reactant multiplicity matrix R (M x S, entries 0..2, row sum <= 2) and a
product matrix P (M x S, entries >= 0); the net change is P - R.

Random networks use numpy's PCG64 generator, seeded explicitly, so the same
seed gives the same network on every machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
import os

import numpy as np

__all__ = [
    "Network", "Workload", "birth_death", "hiv_shaped", "isomerisation",
    "dimerisation", "random_network", "workload_birth_death",
    "workload_hiv_shaped", "workload_random", "batch_networks",
    "tiny_networks", "paper_hiv",
]


@dataclass
class Network:
    """A mass-action reaction network (Sec. 3.2 model format)."""
    name: str
    species: list[str]
    reactants: np.ndarray  # int32 [M, S], 0..2, row sum <= 2
    products: np.ndarray   # int32 [M, S], >= 0
    rates: np.ndarray      # float64 [M], stochastic rate constants c_j >= 0
    x0: np.ndarray         # int32 [S], initial counts >= 0
    # state-dependent rates: (reaction j, species f, slope k, lo, hi) -- the
    # rate of j is min(max(c_j + k x_f, lo), hi)
    modifiers: list = field(default_factory=list)

    @property
    def n_species(self) -> int:
        return int(self.reactants.shape[1])

    @property
    def n_reactions(self) -> int:
        return int(self.reactants.shape[0])

    def with_rates(self, rates) -> "Network":
        return Network(self.name, list(self.species), self.reactants.copy(),
                       self.products.copy(), np.ascontiguousarray(rates, dtype=np.float64),
                       self.x0.copy(), list(self.modifiers))

    def modifier_arrays(self):
        """(f [M] int32, k, lo, hi [M] float64) with f = -1 for unmodified
        reactions, or None when the network has no modifiers."""
        if not self.modifiers:
            return None
        M = self.n_reactions
        f = np.full(M, -1, dtype=np.int32)
        k = np.zeros(M)
        lo = np.zeros(M)
        hi = np.full(M, np.inf)
        for j, sp, slope, a, b in self.modifiers:
            f[j], k[j], lo[j], hi[j] = sp, slope, a, b
        return f, k, lo, hi


@dataclass
class Workload:
    """A network plus the ensemble settings of one run."""
    net: Network
    n_traj: int
    t_end: float
    n_grid: int
    seed: int
    extra: dict = field(default_factory=dict)


def _net(name, species, rxns, rates, x0) -> Network:
    """Build matrices from a list of (reactant dict, product dict)."""
    idx = {s: i for i, s in enumerate(species)}
    M, S = len(rxns), len(species)
    R = np.zeros((M, S), dtype=np.int32)
    P = np.zeros((M, S), dtype=np.int32)
    for j, (rd, pd) in enumerate(rxns):
        for s, v in rd.items():
            R[j, idx[s]] += v
        for s, v in pd.items():
            P[j, idx[s]] += v
    return Network(name, list(species), R, P, np.asarray(rates, dtype=np.float64),
                   np.asarray([x0.get(s, 0) for s in species], dtype=np.int32))


def birth_death(k1: float = 10.0, k2: float = 0.1, x0: int = 0) -> Network:
    """0 -> X (k1), X -> 0 (k2, first order)."""
    return _net("birth_death", ["X"], [({}, {"X": 1}), ({"X": 1}, {})], [k1, k2], {"X": x0})


def hiv_shaped() -> Network:
    """Four-species synthetic immune model (T, I, V, E), ten mass-action reactions."""
    sp = ["T", "I", "V", "E"]
    rx = [
        ({}, {"T": 1}),                       # 0 -> T        10
        ({"T": 1}, {}),                       # T -> 0        0.01
        ({"T": 1, "V": 1}, {"I": 1}),         # T + V -> I    2e-5
        ({"I": 1}, {}),                       # I -> 0        0.5
        ({"I": 1}, {"I": 1, "V": 1}),         # I -> I + V    50
        ({"V": 1}, {}),                       # V -> 0        3
        ({"I": 1, "E": 1}, {"E": 1}),         # I + E -> E    1e-3
        ({"I": 1, "E": 1}, {"I": 1, "E": 2}), # I + E -> I+2E 1e-4
        ({}, {"E": 1}),                       # 0 -> E        1
        ({"E": 1}, {}),                       # E -> 0        0.1
    ]
    rates = [10.0, 0.01, 2e-5, 0.5, 50.0, 3.0, 1e-3, 1e-4, 1.0, 0.1]
    return _net("hiv_shaped", sp, rx, rates, {"T": 1000, "I": 0, "V": 100, "E": 10})


def isomerisation(c1: float = 1.0, c2: float = 0.5, a0: int = 30, b0: int = 10) -> Network:
    """A -> B (c1), B -> A (c2)."""
    return _net("isomerisation", ["A", "B"], [({"A": 1}, {"B": 1}), ({"B": 1}, {"A": 1})],
                [c1, c2], {"A": a0, "B": b0})


def dimerisation(c1: float = 0.3, c2: float = 0.2, c3: float = 0.05, a0: int = 8, b0: int = 5) -> Network:
    """2A -> C (c1), C -> 2A (c2), A + B -> C (c3): exercises both second-order forms."""
    return _net("dimerisation", ["A", "B", "C"],
                [({"A": 2}, {"C": 1}), ({"C": 1}, {"A": 2}), ({"A": 1, "B": 1}, {"C": 1})],
                [c1, c2, c3], {"A": a0, "B": b0, "C": 0})


def random_network(seed: int, n_species: int = 32, n_reactions: int = 128,
                   rate_lo: float = 1e-3, rate_hi: float = 10.0, x0_hi: int = 200) -> Network:
    """Random mass-action network.

    Reaction order uniform in {0, 1, 2}; each reactant is a uniform species pick
    with replacement (two equal picks give a 2X reaction); product count uniform
    in {0, 1, 2}, also uniform picks with replacement; rate log-uniform in
    [rate_lo, rate_hi]; initial counts uniform integers in [0, x0_hi].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    S, M = n_species, n_reactions
    R = np.zeros((M, S), dtype=np.int32)
    P = np.zeros((M, S), dtype=np.int32)
    order = rng.integers(0, 3, size=M)
    for j in range(M):
        for _ in range(int(order[j])):
            R[j, rng.integers(0, S)] += 1
        for _ in range(int(rng.integers(0, 3))):
            P[j, rng.integers(0, S)] += 1
    rates = np.exp(rng.uniform(math.log(rate_lo), math.log(rate_hi), size=M))
    x0 = rng.integers(0, x0_hi + 1, size=S).astype(np.int32)
    return Network(f"random_s{S}_m{M}_seed{seed}", [f"X{i}" for i in range(S)], R, P,
                   rates.astype(np.float64), x0)


def paper_hiv() -> Network:
    """The paper's model of the immune response to HIV (Table 1, Sec. 2.1):
    species U0 (constant source), U, T, Z5, Z4, I5, I4, V5, V4, F; 27
    reactions with the stochastic rates of Sec. 2.1 used as stated (volume
    1).  The bursts I -> 200 V consume the infected cell.  The infectivities
    depend on TNF: beta_R5 = beta - K F (clamped to [0, beta]),
    beta_X4 = beta + K F, gamma_R5/X4 = gamma -/+ K F, as rate modifiers.
    Initial state U0 = 1, U = 200, T = 1000, Z4 = Z5 = 250, V5 = 100."""
    lam, d_uf, d_ut, d_uz, d_t, d_tf = 200.0, 1e-5, 0.129, 0.005, 0.01, 1e-5
    beta, gamma, K = 4e-5, 2e-5, 1e-7
    s1, s2, s3, d_iz, mu, pi, d_i, d_z, d_v = 1e-4, 1e-3, 1e-4, 0.06, 2.5e-3, 200.0, 0.33, 0.01, 2.0
    sp = ["U0", "U", "T", "Z5", "Z4", "I5", "I4", "V5", "V4", "F"]
    rx = [
        ({"U0": 1}, {"U0": 1, "U": 1}, lam),
        ({"U": 1, "F": 1}, {"F": 1}, d_uf),
        ({"U": 1}, {"T": 1}, d_ut),
        ({"U": 1}, {"Z4": 1}, d_uz),
        ({"U": 1}, {"Z5": 1}, d_uz),
        ({"T": 1}, {}, d_t),
        ({"T": 1, "F": 1}, {"F": 1}, d_tf),
        ({"T": 1, "V5": 1}, {"I5": 1}, beta),          # beta_R5
        ({"T": 1, "V4": 1}, {"I4": 1}, beta),          # beta_X4
        ({"Z5": 1, "V5": 1}, {"I5": 1}, gamma),        # gamma_R5
        ({"Z4": 1, "V4": 1}, {"I4": 1}, gamma),        # gamma_X4
        ({"I5": 1}, {"I5": 1, "Z5": 1}, s2),
        ({"I4": 1}, {"I4": 1, "Z4": 1}, s2),
        ({"I5": 1, "Z5": 1}, {"U": 1, "I5": 1, "Z5": 1}, s1),
        ({"I4": 1, "Z4": 1}, {"U": 1, "I4": 1, "Z4": 1}, s1),
        ({"I5": 1, "Z5": 1}, {"Z5": 1}, d_iz),
        ({"I4": 1, "Z4": 1}, {"Z4": 1}, d_iz),
        ({"V5": 1}, {"V4": 1}, mu),
        ({"I5": 1}, {"V5": 200}, pi),
        ({"I4": 1}, {"V4": 200}, pi),
        ({"V4": 1}, {"F": 1, "V4": 1}, s3),
        ({"I5": 1}, {}, d_i),
        ({"I4": 1}, {}, d_i),
        ({"Z5": 1}, {}, d_z),
        ({"Z4": 1}, {}, d_z),
        ({"V5": 1}, {}, d_v),
        ({"V4": 1}, {}, d_v),
    ]
    x0 = {"U0": 1, "U": 200, "T": 1000, "Z4": 250, "Z5": 250, "V5": 100}
    net = _net("paper_hiv", sp, [(a, b) for a, b, _ in rx], [c for _, _, c in rx], x0)
    F = sp.index("F")
    net.modifiers = [(7, F, -K, 0.0, beta), (8, F, K, 0.0, float("inf")),
                     (9, F, -K, 0.0, gamma), (10, F, K, 0.0, float("inf"))]
    return net


def workload_paper_hiv(n_traj: int = 4096, seed: int = 1) -> Workload:
    """The paper's HIV model over 10 days (about 3.8e5 events per trajectory),
    1001-point grid."""
    return Workload(paper_hiv(), n_traj, 10.0, 1001, seed)


def hiv_target_rates(seed: int = 2) -> np.ndarray:
    """Rates of the HIV-shaped model each scaled by exp(U(-0.2, 0.2)), seeded:
    the parameters whose ensemble mean of V is the gradient workload's target."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return hiv_shaped().rates * np.exp(rng.uniform(-0.2, 0.2, size=10))


HIV_TARGET_FILE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                               "hiv_target_v.txt")


def hiv_target_v() -> np.ndarray:
    """The gradient workload's target trajectory: mean V(g) on the 3001-point
    grid of [0, 30] (written by tests/golden/make_hiv_target.py)."""
    with open(HIV_TARGET_FILE) as f:
        vals = [float.fromhex(line.split()[0]) for line in f if line.strip() and not line.startswith("#")]
    return np.array(vals, dtype=np.float64)


def workload_birth_death(n_traj: int = 1000) -> Workload:
    """Birth-death, t_end = 100, 1001-point uniform grid, seed 1."""
    return Workload(birth_death(), n_traj, 100.0, 1001, 1)


def workload_hiv_shaped(n_traj: int = 65536, seed: int = 1) -> Workload:
    """HIV-shaped four-species model, t_end = 30, 3001-point grid."""
    return Workload(hiv_shaped(), n_traj, 30.0, 3001, seed)


def workload_random(n_traj: int = 262144, net_seed: int = 3, seed: int = 1) -> Workload:
    """Random 32-species / 128-reaction network, t_end = 10, 1001-point grid."""
    return Workload(random_network(net_seed), n_traj, 10.0, 1001, seed)


def batch_network(seed: int, traj_lo: int = 1024, traj_hi: int = 65536) -> Workload:
    """One network of the uneven batch, drawn from `seed`: species in [4, 64],
    reactions in [8, 512], trajectory count log-uniform in [traj_lo, traj_hi]
    (rounded), t_end = 10, 501-point grid."""
    rng = np.random.Generator(np.random.PCG64(seed))
    S = int(rng.integers(4, 65))
    M = int(rng.integers(8, 513))
    n = int(round(math.exp(rng.uniform(math.log(traj_lo), math.log(traj_hi)))))
    net = random_network(seed, S, M)
    return Workload(net, n, 10.0, 501, 1, {"seed": seed})


BATCH_SEEDS_FILE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                                "batch_networks.txt")


def batch_seeds() -> list:
    """Accepted network seeds of the batched workload (written by
    tests/golden/make_batch_networks.py: draws whose 16-trajectory pilot
    runs away are rejected)."""
    with open(BATCH_SEEDS_FILE) as f:
        return [int(line) for line in f if line.strip() and not line.startswith("#")]


def batch_networks(n_networks: int = 256, traj_div: int = 1):
    """The uneven batch: the first n_networks accepted seeds, trajectory counts
    divided by traj_div (at least 1)."""
    out = []
    for b, seed in enumerate(batch_seeds()[:n_networks]):
        w = batch_network(seed)
        w = Workload(w.net, max(1, w.n_traj // traj_div), w.t_end, w.n_grid, w.seed, {"index": b, "seed": seed})
        out.append(w)
    return out


def tiny_networks():
    """Small networks whose truncated state space is small enough for an exact
    transient solution (used by the brute-force tests)."""
    return [
        (isomerisation(1.0, 0.5, 6, 3), 2.0),
        (dimerisation(0.3, 0.2, 0.05, 8, 5), 3.0),
        (birth_death(2.0, 0.5, 3), 4.0),
    ]
