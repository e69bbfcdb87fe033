"""Pins for the oracle's likelihood-ratio sensitivities (no GPU).

dL/dc_r is estimated as the mean over trajectories of
  g_r = sum_k u_k Z_r(g_k),  u_k = sum_s w[k][s] (x_s(g_k) - m[k][s]),
  Z_r(t) = N_r(t) / c_r - int_0^t h_r(x(s)) ds
(the score of a mass-action CTMC path).  The estimate is checked against:
  * the birth-death closed forms d mean(t)/dk1 = (1 - e^{-k2 t}) / k2 and
    d mean(t)/dk2 = -(k1/k2^2)(1 - e^{-k2 t}) + (k1/k2) t e^{-k2 t};
  * the derivative of the isomerisation mean A0 p + B0 q in closed form;
  * common-random-number central differences of the oracle's own ensemble
    mean (step 2% of each rate), within max(5 %, 3 combined SE);
each at 3 standard errors of the estimator.
"""
import math

import numpy as np

import oracle
import workloads as W


def _grad(net, N, T, G, seed, w, threads=8):
    r = oracle.run(net, N, T, G, seed, threads=threads)
    mean, _ = oracle.finalize(N, r.S1, r.S2)
    g = oracle.grad(net, N, T, G, seed, w, mean, threads=threads)
    return g.mean(axis=0), g.std(axis=0, ddof=1) / math.sqrt(N), mean


def test_birth_death_gradient_matches_closed_form():
    k1, k2 = 10.0, 0.1
    net = W.birth_death(k1, k2, 0)
    N, T, G = 20000, 20.0, 21
    tg = oracle.uniform_grid(G, T)
    rng = np.random.default_rng(3)
    w = np.zeros((G, 1))
    w[[5, 12, 20], 0] = rng.uniform(0.5, 2.0, size=3)  # L = sum_k w_k mean(g_k)
    est, se, _ = _grad(net, N, T, G, 1, w)
    e = np.exp(-k2 * tg)
    d_k1 = (1 - e) / k2
    d_k2 = -(k1 / k2 ** 2) * (1 - e) + (k1 / k2) * tg * e
    exact = np.array([(w[:, 0] * d_k1).sum(), (w[:, 0] * d_k2).sum()])
    z = np.abs(est - exact) / se
    assert np.all(z < 3.0), (est, exact, se)
    assert se[0] < 0.05 * abs(exact[0])


def test_isomerisation_gradient_matches_closed_form():
    c1, c2, A0, B0 = 1.3, 0.7, 30, 10
    net = W.isomerisation(c1, c2, A0, B0)
    N, T, G = 16000, 3.0, 16
    tg = oracle.uniform_grid(G, T)

    def meanA(a, b):
        k = a + b
        p = (b + a * np.exp(-k * tg)) / k
        q = b * (1.0 - np.exp(-k * tg)) / k
        return A0 * p + B0 * q

    # analytic derivatives of the closed form (complex step: exact to rounding)
    hstep = 1e-30
    dA_dc1 = (meanA(c1 + 1j * hstep, c2)).imag / hstep
    dA_dc2 = (meanA(c1, c2 + 1j * hstep)).imag / hstep
    w = np.zeros((G, 2))
    w[3:, 0] = 1.0  # L = sum over t > 0.5 of mean A
    est, se, _ = _grad(net, N, T, G, 2, w)
    exact = np.array([dA_dc1[3:].sum(), dA_dc2[3:].sum()])
    assert np.all(np.abs(est - exact) / se < 3.0), (est, exact, se)


def test_gradient_matches_common_random_number_differences():
    net = W.hiv_shaped()
    N, T, G = 3000, 6.0, 31
    rng = np.random.default_rng(5)
    w = rng.uniform(-1.0, 1.0, size=(G, 4)) * np.array([1e-3, 1e-1, 1e-2, 1e-1])
    est, se, _ = _grad(net, N, T, G, 4, w, threads=16)
    for r in (0, 4, 5, 8):  # T production, virion burst, virion decay, E production
        h = 0.02 * net.rates[r]
        diffs = []
        for sign in (+1.0, -1.0):
            rates = net.rates.copy()
            rates[r] += sign * h
            rr = oracle.run(net.with_rates(rates), N, T, G, 4, threads=16)
            m, _ = oracle.finalize(N, rr.S1, rr.S2)
            diffs.append((w * m).sum())
        fd = (diffs[0] - diffs[1]) / (2 * h)
        # standard error of the difference quotient by batch means (CRN pairs)
        B = 10
        qs = []
        for b in range(B):
            vals = []
            for sign in (+1.0, -1.0):
                rates = net.rates.copy()
                rates[r] += sign * h
                rr = oracle.run(net.with_rates(rates), N // B, T, G, 4, traj_begin=b * (N // B), threads=16)
                m, _ = oracle.finalize(N // B, rr.S1, rr.S2)
                vals.append((w * m).sum())
            qs.append((vals[0] - vals[1]) / (2 * h))
        se_fd = np.std(qs, ddof=1) / math.sqrt(B)
        se_comb = math.hypot(se[r], se_fd)
        assert abs(est[r] - fd) <= max(0.05 * abs(fd), 3.0 * se_comb), (r, est[r], fd, se[r], se_fd)


def test_gradient_rejects_zero_rates_and_is_zero_without_loss():
    net = W.birth_death(10.0, 0.0, 0)
    try:
        oracle.grad(net, 4, 1.0, 3, 1, np.zeros((3, 1)), np.zeros((3, 1)))
        raise AssertionError("a zero rate must be refused")
    except ValueError:
        pass
    net = W.birth_death(10.0, 0.1, 0)
    g = oracle.grad(net, 50, 5.0, 6, 1, np.zeros((6, 1)), np.zeros((6, 1)))
    assert np.all(g == 0.0)
