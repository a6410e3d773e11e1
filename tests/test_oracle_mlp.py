"""Pins of the oracle's preconditioner network (an extension, not in the
paper): finite differences of the loss gradient, closed forms of the
forward pass, and the identity case (d = 1) reducing to plain L-BFGS."""
import math

import numpy as np
import pytest

from paper_1810_03358_gb300 import synth


def test_mlp_forward_closed_form(oracle_mod):
    w = np.zeros(449)
    w[448] = 0.7  # b2 only
    assert oracle_mod.mlp_forward(w, [1, 2, 3, 4, 5]) == 0.7
    # one hidden unit with weights (1, 0, 0, 0, 0), bias -0.5, output 2
    w[0] = 1.0
    w[320] = -0.5
    w[384] = 2.0
    assert oracle_mod.mlp_forward(w, [1.5, 9, 9, 9, 9]) == pytest.approx(0.7 + 2.0 * 1.0)
    assert oracle_mod.mlp_forward(w, [0.2, 9, 9, 9, 9]) == pytest.approx(0.7)  # ReLU off


def test_mlp_features():
    from oracle import oracle as O
    f = O.mlp_features(0.3, 3.1, 0.05, 32, math.e - 1.0)
    assert np.allclose(f, [0.3, 3.1, 0.05, 0.5, 1.0])


def test_mlp_gradient_finite_differences(oracle_mod):
    rng = np.random.default_rng(3)
    w = rng.normal(scale=0.3, size=449)
    feat = rng.normal(size=(50, 5))
    t = rng.normal(size=50)
    loss, g = oracle_mod.mlp_loss_grad(w, feat, t)
    h = 1e-6
    for k in list(range(0, 449, 17)) + [448, 447, 320, 384]:
        wp = w.copy(); wp[k] += h
        wm = w.copy(); wm[k] -= h
        fd = (oracle_mod.mlp_loss_grad(wp, feat, t)[0] - oracle_mod.mlp_loss_grad(wm, feat, t)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-8), k
    # the loss is the mean squared error of the forward pass
    z = np.array([oracle_mod.mlp_forward(w, f) for f in feat])
    assert loss == pytest.approx(np.mean((z - t) ** 2), rel=1e-12)


def test_identity_network_is_plain_lbfgs(oracle_mod):
    # z = 0 everywhere -> d = exp(0) = 1: the preconditioned run is plain L-BFGS
    s = synth.make_system(40, 41)
    w = np.zeros(449)
    x1, r1 = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS, max_iter=80)
    x2, r2 = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS, max_iter=80, mlp_w=w)
    assert r1["iterations"] == r2["iterations"] and r1["energy"] == r2["energy"]
    assert np.array_equal(x1, x2)


def test_scaled_network_changes_lbfgs(oracle_mod):
    s = synth.make_system(40, 41)
    w = np.zeros(449)
    w[448] = 1.0  # d = e on every atom: H0 scaled by e
    x1, r1 = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS, max_iter=30)
    x2, r2 = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS, max_iter=30, mlp_w=w)
    # a uniform H0 scale leaves normalised directions unchanged in the first
    # two-loop step only in exact arithmetic up to history effects; the runs
    # must both be valid descents
    assert r2["energy"] < oracle_mod.energy(s, s.x)


def _varied_network():
    # per-atom diagonals well away from 1 (a network of random weights)
    w = np.random.default_rng(17).normal(scale=0.4, size=449)
    return w


def test_safeguard_window_one_is_plain_lbfgs(oracle_mod):
    # pc_window = 1 with an unreachable decrease (pc_rel huge) and no
    # gradient floor: the check after the first step (a steepest-descent
    # step, taken before any learned direction) drops the diagonal, so the
    # whole run is plain L-BFGS, bit for bit
    s = synth.make_system(40, 41)
    w = _varied_network()
    x1, r1 = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS, max_iter=60)
    x2, r2 = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS, max_iter=60, mlp_w=w,
                                 pc_window=1, pc_rel=1e300, pc_gfar=0.0)
    assert r1["iterations"] == r2["iterations"] and r1["energy"] == r2["energy"]
    assert np.array_equal(x1, x2)
    # the network does change the run when the safeguard is off
    x3, r3 = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS, max_iter=60, mlp_w=w, pc_window=0)
    assert not np.array_equal(x1, x3)


def test_safeguard_keeps_the_diagonal_while_the_energy_falls(oracle_mod):
    # every 5 steps the energy falls by far more than 1e-12 |E| on a clashing
    # start: the safeguard never fires and the run is the unguarded one
    s = synth.make_system(40, 41)
    w = _varied_network()
    x1, r1 = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS, max_iter=60, mlp_w=w, pc_window=0)
    x2, r2 = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS, max_iter=60, mlp_w=w,
                                 pc_window=5, pc_rel=1e-12, pc_gfar=0.0)
    assert r1["energy"] == r2["energy"] and np.array_equal(x1, x2)


def test_safeguard_needs_a_gradient_far_from_the_tolerance(oracle_mod):
    # the same unreachable decrease, but |grad|_inf must exceed 1e300 times
    # the tolerance: never true, so the diagonal stays in use
    s = synth.make_system(40, 41)
    w = _varied_network()
    x1, r1 = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS, max_iter=60, mlp_w=w, pc_window=0)
    x2, r2 = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS, max_iter=60, mlp_w=w,
                                 pc_window=1, pc_rel=1e300, pc_gfar=1e300)
    assert r1["energy"] == r2["energy"] and np.array_equal(x1, x2)
