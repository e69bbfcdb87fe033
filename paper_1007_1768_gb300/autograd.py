"""torch.autograd.Function over libssa: the ensemble's grid mean and variance
as a differentiable function of the rate constants.

Forward: ssa_ensemble_run (FP64, thread schedule for networks that fit it).
Backward: ssa_ensemble_grad replays the same trajectories from their Philox
counters and returns the likelihood-ratio estimate of dL/drates from
dL/dmean.  Gradients through the variance are not provided: a backward call
with a nonzero grad for var raises.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as _b


class SSAEnsembleFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rates, reactants, products, x0, n_traj, t_end, n_grid, seed, device, opt_kw):
        model = _b.Model(reactants, products, rates.detach().to("cpu", torch.float64).numpy(), x0)
        r = _b.ensemble_run(model, n_traj, t_end, n_grid, seed, device=device, want_sums=False, per_traj=True,
                            **opt_kw)
        ctx.model = model
        ctx.call = (n_traj, t_end, n_grid, seed, device, opt_kw)
        ctx.rates_meta = (rates.device, rates.dtype)
        ctx.traj_events = r.traj_events  # the backward replays the longest trajectories first
        ctx.save_for_backward(r.mean)
        ctx.last_se = None
        return r.mean, r.var

    @staticmethod
    def backward(ctx, grad_mean, grad_var):
        if grad_var is not None and bool((grad_var != 0).any()):
            raise RuntimeError("gradients through the variance are not provided; use the mean")
        (mean,) = ctx.saved_tensors
        n_traj, t_end, n_grid, seed, device, opt_kw = ctx.call
        if grad_mean is None:
            grad_mean = torch.zeros_like(mean)
        # the model stays open until the graph is freed (Model.__del__), so a
        # second backward through a retained graph replays it again
        g, se, _ = _b.ensemble_grad(ctx.model, n_traj, t_end, n_grid, seed, grad_mean.contiguous(), mean,
                                    device=device, traj_events=ctx.traj_events, **opt_kw)
        dev, dt = ctx.rates_meta
        SSAEnsembleFunction.last_standard_error = se.to(dev, dt)
        return g.to(dev, dt), None, None, None, None, None, None, None, None, None


def ssa_ensemble(rates: torch.Tensor, network, n_traj: int, t_end: float, n_grid: int, seed: int,
                 device="cuda:0", **opt_kw):
    """(mean [G, S], var [G, S]) on `device` for the network's structure
    (reactants, products, x0) at `rates` ([M], differentiable).  After a
    backward pass, SSAEnsembleFunction.last_standard_error holds the standard
    errors of the rate gradient."""
    R = np.ascontiguousarray(network.reactants, dtype=np.int32)
    P = np.ascontiguousarray(network.products, dtype=np.int32)
    x0 = np.ascontiguousarray(network.x0, dtype=np.int32)
    return SSAEnsembleFunction.apply(rates, R, P, x0, int(n_traj), float(t_end), int(n_grid), int(seed), device,
                                     dict(opt_kw))
