"""GPU parity of state-dependent rates (rate modifiers, the paper's
TNF-dependent infectivities) and of the paper's HIV model (Table 1) against
the oracle in the warp schedule, bit for bit; the dependency graph must
recompute a modified reaction when its modifier species changes."""
import numpy as np
import pytest

import oracle
import paper_1007_1768_gb300 as ssa
import workloads as W

pytestmark = pytest.mark.gpu
W32 = oracle.SCHEDULE_W32


def _gpu(net, n, T, G, seed, **kw):
    model = ssa.Model.from_network(net)
    try:
        return ssa.ensemble_run(model, n, T, G, seed, per_traj=True, **kw)
    finally:
        model.close()


def _same(g, net, n, T, G, seed, **kw):
    r = oracle.run(net, n, T, G, seed, per_traj=True, threads=16, schedule=W32, **kw)
    assert np.array_equal(g.traj_hash, r.traj_hash) and np.array_equal(g.traj_events, r.traj_events)
    assert np.array_equal(g.sum1, r.S1) and np.array_equal(g.sum2, r.S2)


def test_modifier_species_that_changes():
    # X -> 0 at rate 0.05 + 0.02 Y (clamped to [0, 0.3]); 0 -> Y (1.5); Y -> 0 (0.1)
    R = np.array([[1, 0], [0, 0], [0, 1]], np.int32)
    P = np.array([[0, 0], [0, 1], [0, 0]], np.int32)
    net = W.Network("mod_dep", ["X", "Y"], R, P, np.array([0.05, 1.5, 0.1]), np.array([200, 0], np.int32))
    net.modifiers = [(0, 1, 0.02, 0.0, 0.3)]
    g = _gpu(net, 300, 20.0, 41, 3)
    _same(g, net, 300, 20.0, 41, 3)
    # a negative slope clamped at 0 once Y is large
    net.modifiers = [(0, 1, -0.01, 0.0, 1.0)]
    g = _gpu(net, 300, 20.0, 41, 4)
    _same(g, net, 300, 20.0, 41, 4)


def test_paper_hiv_model_bit_exact():
    net = W.paper_hiv()
    g = _gpu(net, 24, 0.3, 31, 5)
    _same(g, net, 24, 0.3, 31, 5)
    assert g.events > 24 * 100


def test_modified_model_in_an_fp64_batch_and_avg_xy():
    net = W.paper_hiv()
    models = [ssa.Model.from_network(net), ssa.Model.from_network(W.hiv_shaped())]
    batch = ssa.Batch(models, [16, 40], [0.2, 5.0], [21, 51], precision="fp64")
    outs, _ = batch.launch(7, want_sums=True)
    r = oracle.run(net, 16, 0.2, 21, 7, stream=0, schedule=W32, threads=16)
    assert np.array_equal(outs[0]["sum1"], r.S1) and np.array_equal(outs[0]["sum2"], r.S2)
    batch.close()
    t, m, q, U = ssa.ensemble_avg_xy(models[0], 6, 0.05, 2, 50)
    ot, om, oq, oU = oracle.avg_xy(net, 6, 0.05, 2, 50, schedule=W32)
    assert U == oU and np.array_equal(t, ot) and np.array_equal(m, om) and np.array_equal(q, oq)
    for mdl in models:
        mdl.close()
