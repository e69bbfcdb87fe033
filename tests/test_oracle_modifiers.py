"""Pins for the oracle's rate modifiers (state-dependent rates, the paper's
TNF-dependent infectivities, Sec. 2.1): rate_j = min(max(c_j + k x_f, lo), hi).

  * slope 0 leaves the mass-action model unchanged, bit for bit;
  * X -> 0 with rate c + k Y, Y a species no reaction changes, is a pure
    death process with rate lambda = clamp(c + k Y): X(t) ~ Bin(x0, e^{-lambda t}),
    checked in the unclamped case and at both clamps (lo: no decay at all,
    hi: the capped rate);
  * the paper's HIV model: the modified infectivities follow F.
"""
import numpy as np

import oracle
import workloads as W


def _decay(c, k, lo, hi, Y, x0=40):
    R = np.array([[1, 0]], np.int32)
    P = np.array([[0, 0]], np.int32)
    net = W.Network("decay_mod", ["X", "Y"], R, P, np.array([c]), np.array([x0, Y], np.int32))
    net.modifiers = [(0, 1, k, lo, hi)]
    return net


def test_zero_slope_is_mass_action():
    base = W.hiv_shaped()
    mod = base.with_rates(base.rates)
    mod.modifiers = [(2, 2, 0.0, 0.0, np.inf), (4, 0, 0.0, 0.0, np.inf)]
    a = oracle.run(base, 50, 30.0, 31, 3, per_traj=True)
    b = oracle.run(mod, 50, 30.0, 31, 3, per_traj=True)
    assert np.array_equal(a.traj_hash, b.traj_hash) and np.array_equal(a.S2, b.S2)


def _check_binomial(net, lam, N=20000, T=3.0, G=13):
    r = oracle.run(net, N, T, G, 5, threads=8)
    mean, var = oracle.finalize(N, r.S1, r.S2)
    g = oracle.uniform_grid(G, T)
    x0 = int(net.x0[0])
    p = np.exp(-lam * g)
    mu, sig2 = x0 * p, x0 * p * (1 - p)
    assert np.all(mean[:, 1] == net.x0[1])  # Y never changes
    se = np.sqrt(np.maximum(sig2, 1e-300) / N)
    inner = sig2 > 0
    assert np.all(np.abs(mean[inner, 0] - mu[inner]) / se[inner] < 4.5)
    return r


def test_modified_decay_rate_closed_form():
    _check_binomial(_decay(0.5, 0.1, 0.0, np.inf, 3), 0.8)           # 0.5 + 0.3
    _check_binomial(_decay(0.5, 1.0, 0.0, 1.0, 3), 1.0)              # capped at hi
    r = oracle.run(_decay(0.5, -0.3, 0.0, np.inf, 3), 100, 3.0, 4, 5)  # 0.5 - 0.9 < 0: clamped to lo = 0
    assert r.events == 0 and np.all(r.S1[:, 0] == 100 * 40)


def test_paper_hiv_infectivities_follow_tnf():
    net = W.paper_hiv()
    names = net.species
    F = names.index("F")
    assert net.n_reactions == 27 and net.n_species == 10
    # with a large F the R5 infectivity is clamped to 0: no T + V5 -> I5 events
    heavy = net.with_rates(net.rates)
    heavy.x0 = net.x0.copy()
    heavy.x0[F] = 1000  # beta - K F = 4e-5 - 1e-4 < 0, gamma likewise
    heavy.x0[names.index("V5")] = 1000
    # (unclamped, T + V5 -> I5 would fire ~20 times in 0.5 days)
    rt, rj, _, _, ne = oracle.trace(heavy, 0, 0.5, 1, 3, grid=[0.5], schedule=oracle.SCHEDULE_W32,
                                    record_max=10 ** 6)
    assert ne > 0 and not np.any((rj == 7) | (rj == 9))
    rt, rj, _, _, ne = oracle.trace(net, 0, 0.5, 1, 3, grid=[0.5], schedule=oracle.SCHEDULE_W32,
                                    record_max=10 ** 6)
    assert np.any(rj == 7)  # without F the infection of T by V5 happens
