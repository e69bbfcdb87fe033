"""GPU checks of the likelihood-ratio rate gradient (ssa_ensemble_grad) and
its torch.autograd.Function.

(1) Parity with the oracle, per trajectory.  The kernel replays the same
    trajectories and forms the same score in another association order
    (B_r = Z_r + h_r t updated at events, interval sums from grid prefix
    sums), so the contributions agree to rounding: each is a sum of products
    of FP64 values whose magnitudes are bounded by the trajectory's largest
    |N_r / c_r|, integral and grid-weight sums; a relative tolerance of
    1e-9 of the largest contribution of the same rate covers the few hundred
    rounding steps of a trajectory with wide margin (FP64 unit roundoff is
    1.1e-16).
(2) The birth-death closed form of d mean / d k1 and d mean / d k2 within
    3 standard errors at 1,048,576 trajectories.
(3) Common-random-number central differences (rate +- 2 %) of the HIV-shaped
    loss sum_g (mean V(g) - target_g)^2 within max(5 % of the difference
    quotient, 3 combined standard errors), for all ten rates.
(4) The autograd path gives the same numbers as the direct call.
"""
import math

import numpy as np
import pytest

import oracle
import paper_1007_1768_gb300 as ssa
import workloads as W

pytestmark = pytest.mark.gpu


def _forward(net, n, T, G, seed, grid=None, **kw):
    model = ssa.Model.from_network(net)
    r = ssa.ensemble_run(model, n, T, G, seed, grid=grid, **kw)
    model.close()
    return r


def _grad(net, n, T, G, seed, w, mean, grid=None, per_traj=True, **kw):
    model = ssa.Model.from_network(net)
    try:
        return ssa.ensemble_grad(model, n, T, G, seed, w, mean, grid=grid, per_traj=per_traj, **kw)
    finally:
        model.close()


def _parity(net, n, T, G, seed, grid=None, max_events=0, wscale=None):
    rng = np.random.default_rng(seed)
    Gn = G if grid is None else len(grid)
    f = _forward(net, n, T, Gn, seed, grid=grid, max_events=max_events)
    w = rng.uniform(-1.0, 1.0, size=(Gn, net.n_species))
    if wscale is not None:
        w = w * wscale
    g, se, traj = _grad(net, n, T, Gn, seed, w, f.mean, grid=grid, max_events=max_events)
    og = oracle.grad(net, n, T, Gn, seed, w, f.mean, grid=grid, threads=16,
                     max_events=max_events if max_events > 0 else oracle.MAX_EVENTS)
    scale = np.abs(og).max(axis=0) + 1e-300
    err = np.abs(traj.T - og).max(axis=0)
    assert np.all(err <= 1e-9 * scale), (err / scale)
    assert np.allclose(g, og.mean(axis=0), rtol=1e-9, atol=1e-12 * scale.max())
    assert np.allclose(se, og.std(axis=0, ddof=1) / math.sqrt(n), rtol=1e-6)
    return g


def test_parity_hiv_shaped_and_small_networks():
    _parity(W.hiv_shaped(), 300, 30.0, 301, 5, wscale=np.array([1e-3, 1e-1, 1e-2, 1e-1]))
    _parity(W.birth_death(), 257, 50.0, 101, 3)
    _parity(W.isomerisation(1.3, 0.7, 30, 10), 200, 3.0, 31, 4)
    _parity(W.random_network(88, n_species=6, n_reactions=12, x0_hi=40), 150, 1.0, 41, 6, max_events=20000)


def test_parity_explicit_grid_truncation_and_absorbing():
    net = W.hiv_shaped()
    rt, _, _, _, _ = oracle.trace(net, 0, 30.0, 2, seed=9)
    grid = np.unique(np.concatenate([[0.0], rt[:40], np.linspace(0.5, 30.0, 50)]))
    _parity(net, 120, 30.0, 0, 9, grid=grid, wscale=np.array([1e-3, 1e-1, 1e-2, 1e-1]))
    _parity(net, 90, 30.0, 301, 1, max_events=7, wscale=np.array([1e-3, 1e-1, 1e-2, 1e-1]))
    death = W.Network("death", ["X"], np.array([[1]], np.int32), np.array([[0]], np.int32), np.array([2.0]),
                      np.array([5], np.int32))
    _parity(death, 64, 50.0, 51, 3)


def test_work_order_from_event_counts_changes_nothing():
    """The forward's event counts only reorder the replay (longest first,
    used when the ensemble is several times the resident threads: 240,000
    trajectories here): the gradient, its standard error and every
    per-trajectory contribution are the same bits, with host and with device
    buffers, also for a nonsense order hint and for an ensemble below the
    threshold."""
    import torch
    net = W.hiv_shaped()
    n, G = 240000, 301
    model = ssa.Model.from_network(net)
    try:
        f = ssa.ensemble_run(model, n, 30.0, G, 5, per_traj=True)
        w = np.zeros((G, 4))
        w[:, 2] = 1e-2
        g0, se0, t0 = ssa.ensemble_grad(model, n, 30.0, G, 5, w, f.mean, per_traj=True)
        g1, se1, t1 = ssa.ensemble_grad(model, n, 30.0, G, 5, w, f.mean, per_traj=True, traj_events=f.traj_events)
        rev = np.arange(n, dtype=np.int64)[::-1].copy()
        g2, se2, t2 = ssa.ensemble_grad(model, n, 30.0, G, 5, w, f.mean, per_traj=True, traj_events=rev)
        gd, sed, td = ssa.ensemble_grad(model, n, 30.0, G, 5, torch.as_tensor(w), torch.as_tensor(f.mean),
                                        device="cuda:0", per_traj=True, traj_events=torch.as_tensor(f.traj_events))
        for g, se, t in ((g1, se1, t1), (g2, se2, t2), (gd.cpu().numpy(), sed.cpu().numpy(), td.cpu().numpy())):
            assert np.array_equal(g, g0) and np.array_equal(se, se0) and np.array_equal(t, t0)
        f3 = ssa.ensemble_run(model, 3000, 30.0, G, 6, per_traj=True)
        a3 = ssa.ensemble_grad(model, 3000, 30.0, G, 6, w, f3.mean, per_traj=True)
        b3 = ssa.ensemble_grad(model, 3000, 30.0, G, 6, w, f3.mean, per_traj=True, traj_events=f3.traj_events)
        assert all(np.array_equal(x, y) for x, y in zip(a3, b3))
    finally:
        model.close()


def test_repeatable_and_refusals():
    net = W.hiv_shaped()
    f = _forward(net, 2000, 30.0, 301, 7)
    w = np.ones((301, 4)) * 1e-3
    a = _grad(net, 2000, 30.0, 301, 7, w, f.mean)[0]
    b = _grad(net, 2000, 30.0, 301, 7, w, f.mean)[0]
    assert np.array_equal(a, b)
    with pytest.raises(ssa.SSAError) as e:
        _grad(W.birth_death(10.0, 0.0), 10, 1.0, 3, 1, np.zeros((3, 1)), np.zeros((3, 1)))
    assert e.value.status == ssa.binding.SSA_EUNSUPPORTED
    with pytest.raises(ssa.SSAError) as e:
        _grad(W.random_network(3), 10, 1.0, 3, 1, np.zeros((3, 32)), np.zeros((3, 32)))
    assert e.value.status == ssa.binding.SSA_EUNSUPPORTED


def test_birth_death_closed_form_within_three_standard_errors():
    k1, k2 = 10.0, 0.1
    net = W.birth_death(k1, k2, 0)
    N, T, G = 1 << 20, 20.0, 21
    f = _forward(net, N, T, G, 11)
    tg = oracle.uniform_grid(G, T)
    w = np.zeros((G, 1))
    w[[4, 10, 20], 0] = [0.5, 1.0, 2.0]
    g, se, _ = _grad(net, N, T, G, 11, w, f.mean, per_traj=False)
    e = np.exp(-k2 * tg)
    exact = np.array([(w[:, 0] * (1 - e) / k2).sum(),
                      (w[:, 0] * (-(k1 / k2 ** 2) * (1 - e) + (k1 / k2) * tg * e)).sum()])
    z = np.abs(g - exact) / se
    print("birth-death: grad", g, "exact", exact, "z", z)
    assert np.all(z < 3.0)


def _hiv_loss_grad(rates, N, seed, per_traj=False):
    net = W.hiv_shaped().with_rates(rates)
    target = W.hiv_target_v()
    f = _forward(net, N, 30.0, 3001, seed)
    w = np.zeros((3001, 4))
    w[:, 2] = 2.0 * (f.mean[:, 2] - target)
    loss = float(((f.mean[:, 2] - target) ** 2).sum())
    g, se, _ = _grad(net, N, 30.0, 3001, seed, w, f.mean, per_traj=per_traj)
    return loss, g, se


def test_hiv_gradient_matches_crn_central_differences():
    base = W.hiv_shaped().rates
    N, seed = 131072, 3
    _, g, se = _hiv_loss_grad(base, N, seed)
    target = W.hiv_target_v()
    B = 16
    for r in range(10):
        h = 0.02 * base[r]
        q = []
        for b in range(B):  # batch means over shards of the same random numbers
            vals = []
            for sign in (+1.0, -1.0):
                rates = base.copy()
                rates[r] += sign * h
                f = _forward(W.hiv_shaped().with_rates(rates), N // B, 30.0, 3001, seed, traj_offset=b * (N // B))
                vals.append(f.sum1[:, 2].astype(np.float64))
            q.append(vals)
        # full-ensemble difference quotient of the loss, and the SE of its linearisation
        s_plus = sum(v[0] for v in q) / N
        s_minus = sum(v[1] for v in q) / N
        fd = (((s_plus - target) ** 2).sum() - ((s_minus - target) ** 2).sum()) / (2 * h)
        mid = 0.5 * (s_plus + s_minus)
        lin = [(2.0 * (mid - target) * (v[0] - v[1]) / (N // B) / (2 * h)).sum() for v in q]
        se_fd = np.std(lin, ddof=1) / math.sqrt(B)
        tol = max(0.05 * abs(fd), 3.0 * math.hypot(se[r], se_fd))
        print(f"rate {r}: LR {g[r]:.6g} +- {se[r]:.3g}, FD {fd:.6g} +- {se_fd:.3g}")
        assert abs(g[r] - fd) <= tol, (r, g[r], fd, se[r], se_fd)


def test_autograd_function_matches_direct_call():
    import torch
    from paper_1007_1768_gb300.autograd import SSAEnsembleFunction, ssa_ensemble
    net = W.hiv_shaped()
    target = torch.as_tensor(W.hiv_target_v(), device="cuda:0")
    rates = torch.tensor(net.rates, dtype=torch.float64, requires_grad=True)
    mean, var = ssa_ensemble(rates, net, 8192, 30.0, 3001, 5)
    loss = ((mean[:, 2] - target) ** 2).sum()
    loss.backward()
    _, g, se = _hiv_loss_grad(net.rates, 8192, 5)
    assert np.array_equal(rates.grad.numpy(), g)
    assert np.array_equal(SSAEnsembleFunction.last_standard_error.numpy(), se)
    # gradients through the variance are refused
    rates2 = torch.tensor(net.rates, dtype=torch.float64, requires_grad=True)
    mean2, var2 = ssa_ensemble(rates2, net, 256, 30.0, 301, 5)
    with pytest.raises(RuntimeError):
        var2.sum().backward()


def test_autograd_second_backward_through_a_retained_graph():
    import torch
    from paper_1007_1768_gb300.autograd import ssa_ensemble
    net = W.hiv_shaped()
    target = torch.as_tensor(W.hiv_target_v(), device="cuda:0")
    rates = torch.tensor(net.rates, dtype=torch.float64, requires_grad=True)
    mean, _ = ssa_ensemble(rates, net, 1024, 30.0, 3001, 6)
    loss = ((mean[:, 2] - target) ** 2).sum()
    loss.backward(retain_graph=True)
    g1 = rates.grad.clone()
    rates.grad = None
    loss.backward()
    # the replay is deterministic: the same gradient, bit for bit
    assert torch.equal(rates.grad, g1)

