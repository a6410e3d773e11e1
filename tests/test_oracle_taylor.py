"""Pins of the oracle's linearised far-field Coulomb rows (Section 3's
construction for the gradient-free moves): exact at the current position
and without far atoms, second-order in the displacement, inside Taylor's
remainder bound, and the moves with an infinite radius are the exact ones."""
import numpy as np
import pytest

from paper_1810_03358_gb300 import synth


def test_no_far_atoms_is_the_exact_row(oracle_mod):
    s = synth.make_system(60, 901)
    rng = np.random.default_rng(0)
    for i in (0, 17, 59):
        p = s.x[i] + rng.normal(scale=0.1, size=3)
        exact = oracle_mod.row_energy(s, s.x, i, p)
        assert oracle_mod.row_energy_taylor(s, s.x, i, p, 1e30) == exact


@pytest.mark.parametrize("r_far", [3.0, 6.0, 10.0])
def test_exact_at_the_current_position(oracle_mod, r_far):
    s = synth.make_system(120, 902)
    for i in (3, 60, 119):
        exact = oracle_mod.row_energy(s, s.x, i, s.x[i])
        approx = oracle_mod.row_energy_taylor(s, s.x, i, s.x[i], r_far)
        assert abs(approx - exact) <= 1e-12 * abs(exact)


def coulomb_far(s, i, r_far):
    d = np.linalg.norm(s.x - s.x[i], axis=1)
    far = (d >= r_far) & (np.arange(len(d)) != i)
    return far, d


@pytest.mark.parametrize("i", [5, 70, 140])
def test_second_order_error_and_remainder_bound(oracle_mod, i):
    s = synth.make_system(150, 903)
    r_far = 6.0
    far, d = coulomb_far(s, i, r_far)
    assert far.sum() > 10
    u = np.random.default_rng(i).normal(size=3)
    u /= np.linalg.norm(u)
    errs = []
    for h in (0.05, 0.025, 0.0125):
        p = s.x[i] + h * u
        err = oracle_mod.row_energy_taylor(s, s.x, i, p, r_far) - oracle_mod.row_energy(s, s.x, i, p)
        # Taylor's remainder for C q_i q_j / r: |1/2 delta^T H delta| with
        # |H| <= 2 / r^3 on the segment, r >= r0 - h
        bound = np.sum(s.coulomb_c * np.abs(s.charge[i] * s.charge[far]) * h * h / (d[far] - h) ** 3)
        assert abs(err) <= bound
        errs.append(err)
    # halving the displacement quarters the error (first-order expansion)
    for a, b in zip(errs, errs[1:]):
        assert 3.7 < a / b < 4.3


def test_moves_with_infinite_radius_are_exact(oracle_mod):
    s = synth.make_system(40, 904)
    kw = dict(method=oracle_mod.GRADFREE, max_iter=120, gtol_inf=1e-9, seed=8, gradfree_delta=0.05)
    xa, ra = oracle_mod.minimize(s, s.x, **kw)
    xb, rb = oracle_mod.minimize(s, s.x, gradfree_taylor_r=1e30, **kw)
    assert np.array_equal(xa, xb) and ra["energy"] == rb["energy"]
