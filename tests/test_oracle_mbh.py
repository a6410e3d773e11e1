"""Pins of the oracle's monotonic basin hopping (the construction of Wales
and Doye that Section 2 mentions, monotonic form: perturb the best point,
minimize locally, keep the result when it is lower), with no GPU."""
import numpy as np
import pytest

from paper_1810_03358_gb300 import synth


def tilted_double_well(x, want):
    f = (x[0] ** 2 - 1.0) ** 2 + 0.3 * x[0]
    return f, (np.array([4.0 * x[0] * (x[0] ** 2 - 1.0) + 0.3]) if want else None)


def test_escapes_the_shallow_well(oracle_mod):
    # f = (x^2 - 1)^2 + 0.3 x: stationary points are the roots of
    # 4x^3 - 4x + 0.3 = 0; the local minimizer from 1.2 stops at the shallow
    # minimum, basin hopping (steps of up to 2.5) reaches the deep one
    roots = np.sort(np.roots([4.0, 0.0, -4.0, 0.3]).real)
    deep, shallow = roots[0], roots[2]
    xl, rl = oracle_mod.minimize_fn(tilted_double_well, np.array([1.2]), method=oracle_mod.LBFGS,
                                    gtol_inf=1e-10)
    assert xl[0] == pytest.approx(shallow, abs=1e-8)
    for seed in (1, 2, 3):
        xo, r, acc = oracle_mod.basin_hop_fn(tilted_double_well, np.array([1.2]), 20, 2.5, seed,
                                             method=oracle_mod.LBFGS, gtol_inf=1e-10)
        assert xo[0] == pytest.approx(deep, abs=1e-8)
        assert acc >= 1 and r["status_name"] in ("ok", "linesearch")  # 1e-10 is near the rounding floor
        assert r["energy"] == pytest.approx(tilted_double_well(xo, False)[0], abs=1e-15)


def test_zero_hops_is_the_local_minimizer(oracle_mod):
    s = synth.make_system(30, 51)
    xl, rl = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS)
    xb, rb, acc = oracle_mod.basin_hop(s, s.x, 0, 0.5, 7, method=oracle_mod.LBFGS)
    assert acc == 0 and np.array_equal(xl, xb)
    assert rb["energy"] == rl["energy"] and rb["iterations"] == rl["iterations"]


def test_perturbation_and_acceptance_restated(oracle_mod):
    # with no local steps (max_iter = 0) every hop is one perturbation of the
    # best point; on f = |x|^2 the kept point is rebuilt here from the
    # published SplitMix64 stream (pinned by the golden values):
    # trial_k = best_k + step (2u - 1), u = (z >> 11) 2^-53, z = SM64(seed,
    # h n + k), kept when |trial|^2 < |best|^2
    n, hops, step, seed = 5, 40, 0.7, 99
    x0 = np.array([0.9, -0.4, 0.3, 1.1, -0.8])
    fg = lambda x, want: (float(x @ x), 2.0 * x if want else None)
    xo, r, acc = oracle_mod.basin_hop_fn(fg, x0, hops, step, seed, method=oracle_mod.GD, max_iter=0,
                                         gtol_inf=1e-12)
    best, kept = x0.copy(), 0
    for h in range(hops):
        u = np.array([(oracle_mod.splitmix64(seed, h * n + k) >> 11) * 2.0 ** -53 for k in range(n)])
        trial = best + step * (2.0 * u - 1.0)
        if trial @ trial < best @ best:
            best, kept = trial, kept + 1
    assert acc == kept > 0
    assert np.array_equal(xo, best)
    assert r["energy"] == best @ best


def test_force_field_hops_are_monotone_and_valid(oracle_mod):
    s = synth.make_system(40, 52)
    xl, rl = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS)
    xb, rb, acc = oracle_mod.basin_hop(s, s.x, 6, 0.4, 11, method=oracle_mod.LBFGS)
    assert rb["status_name"] == "ok"
    assert rb["energy"] <= rl["energy"]
    e, g = oracle_mod.energy_grad(s, xb)
    assert e == pytest.approx(rb["energy"], rel=1e-12)
    assert np.abs(g).max() < 0.1
