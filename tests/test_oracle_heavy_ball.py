"""Pins of the oracle's heavy-ball method (Section 4, Eq. 8, constant alpha
and beta): the beta = 0 case is gradient descent with a fixed step (closed
form on a quadratic), a scalar quadratic follows the two-term linear
recurrence's closed form, and Polyak's parameters give his rate."""
import numpy as np
import pytest

from tests.test_oracle_minimizers import quad_fg, spd


def test_beta_zero_is_fixed_step_descent(oracle_mod):
    A, b, lam = spd(10, 20.0, 11)
    xs = np.linalg.solve(A, b)
    alpha = 1.0 / lam[-1]
    x0 = np.zeros(10)
    xo, r = oracle_mod.minimize_fn(quad_fg(A, b), x0, method=oracle_mod.HB, gtol_inf=1e-14, max_iter=12,
                                   hb_alpha=alpha, hb_beta=0.0)
    M = np.eye(10) - alpha * A
    ref = xs + np.linalg.matrix_power(M, 12) @ (x0 - xs)
    assert r["iterations"] == 12
    assert np.abs(xo - ref).max() < 1e-12


@pytest.mark.parametrize("alpha,beta", [(0.3, 0.5), (0.9, 0.2), (0.1, 0.9)])
def test_scalar_quadratic_closed_form(oracle_mod, alpha, beta):
    # f = a x^2 / 2: x_{k+1} = (1 + beta - alpha a) x_k - beta x_{k-1},
    # x_{-1} = x_0; x_k = c1 z1^k + c2 z2^k with the roots of
    # z^2 - (1 + beta - alpha a) z + beta = 0
    a, x0, N = 1.7, 2.0, 15
    A = np.array([[a]])
    z1, z2 = np.roots([1.0, -(1.0 + beta - alpha * a), beta])
    x1 = x0 - alpha * a * x0
    c2 = (x1 - z1 * x0) / (z2 - z1)
    c1 = x0 - c2
    ref = (c1 * z1 ** N + c2 * z2 ** N).real
    xo, r = oracle_mod.minimize_fn(quad_fg(A, np.zeros(1)), np.array([x0]), method=oracle_mod.HB,
                                   gtol_inf=1e-300, max_iter=N, hb_alpha=alpha, hb_beta=beta)
    assert r["iterations"] == N
    assert xo[0] == pytest.approx(ref, rel=1e-10, abs=1e-14)


def test_polyak_parameters_rate(oracle_mod):
    # alpha = 4 / (sqrt L + sqrt mu)^2, beta = ((sqrt L - sqrt mu)/(sqrt L + sqrt mu))^2
    # converge at rate (sqrt kappa - 1) / (sqrt kappa + 1) per step (Polyak 1964)
    A, b, lam = spd(12, 100.0, 12)
    mu, L = lam[0], lam[-1]
    alpha = 4.0 / (np.sqrt(L) + np.sqrt(mu)) ** 2
    beta = ((np.sqrt(L) - np.sqrt(mu)) / (np.sqrt(L) + np.sqrt(mu))) ** 2
    rho = (np.sqrt(L / mu) - 1.0) / (np.sqrt(L / mu) + 1.0)
    xs = np.linalg.solve(A, b)
    errs = []
    for N in (100, 150):
        xo, r = oracle_mod.minimize_fn(quad_fg(A, b), np.zeros(12), method=oracle_mod.HB, gtol_inf=1e-300,
                                       max_iter=N, hb_alpha=alpha, hb_beta=beta)
        errs.append(np.linalg.norm(xo - xs))
    rate = (errs[1] / errs[0]) ** (1.0 / 50)
    assert rate <= rho * 1.05
    assert rate >= rho * 0.8


def test_invalid_parameters(oracle_mod):
    A, b, _ = spd(4, 5.0, 13)
    _, r = oracle_mod.minimize_fn(quad_fg(A, b), np.zeros(4), method=oracle_mod.HB, hb_alpha=0.0)
    assert r["status_name"] == "bad_arg"


def test_heavy_ball_stops_at_last_finite_iterate(oracle_mod):
    # an objective that turns non-finite at its 6th gradient evaluation: the
    # run stops there and returns the 5th iterate (the last finite one) with
    # its energy, not the failing point
    A = np.diag([1.0, 4.0, 9.0])
    calls = {"n": 0}
    iterates = []

    def fg(x, want):
        calls["n"] += 1
        if calls["n"] >= 6:
            return float("nan"), np.full(3, np.nan)
        iterates.append(x.copy())
        return 0.5 * x @ A @ x, A @ x

    x0 = np.array([1.0, -2.0, 0.5])
    xo, r = oracle_mod.minimize_fn(fg, x0, method=oracle_mod.HB, hb_alpha=0.05, hb_beta=0.3,
                                   gtol_inf=1e-12, max_iter=100)
    assert r["status_name"] == "nonfinite"
    assert r["iterations"] == 4  # x^1 .. x^4 accepted; x^5 (6th call) failed
    assert np.array_equal(xo, iterates[-1])
    assert r["energy"] == 0.5 * iterates[-1] @ A @ iterates[-1]
