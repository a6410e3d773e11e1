"""Pins of the oracle's line searches (Algorithms 5, 6) and minimizers
(Algorithms 1-4, Eq. 4, the gradient-free parab moves) against textbook
results on functions with known answers, with no GPU."""
import math

import numpy as np
import pytest

from paper_1810_03358_gb300 import synth


# ------------------------------ line searches ------------------------------

def test_ls_par_exact_on_parabola(oracle_mod):
    # phi(h) = a (h - hs)^2 + c: the G0 parabola through f(0), f'(0), f(h0) is
    # the function itself, so the first fit lands on hs (Section 5.2, Alg. 6).
    a, hs, c = 3.0, 0.37, -2.0
    phi = lambda h: a * (h - hs) ** 2 + c
    f0, slope = phi(0.0), -2 * a * hs
    h, f, calls = oracle_mod.ls_par(phi, f0, slope, 0.1, K=2, g0=1)
    assert calls[0] == 0.1
    assert calls[1] == pytest.approx(hs, rel=1e-12)
    assert len(calls) == 3  # K = 2: h0, the G0 vertex, one refinement
    assert h == pytest.approx(hs, rel=1e-12) and f == pytest.approx(c, rel=1e-12)


def test_ls_par_g0_false_symmetric_points(oracle_mod):
    a, hs, c = 0.5, -0.04, 1.0
    phi = lambda h: a * (h - hs) ** 2 + c
    h, f, calls = oracle_mod.ls_par(phi, phi(0.0), 0.0, 0.2, K=2, g0=0)
    assert calls[:2] == [-0.1, 0.1]
    assert calls[2] == pytest.approx(hs, abs=1e-14)
    assert h == pytest.approx(hs, abs=1e-14)


def test_ls_par_more_refinements(oracle_mod):
    # a non-quadratic convex function: K refinements must not increase f
    phi = lambda h: math.cosh(3 * (h - 0.8)) + 0.1 * h ** 4
    f0 = phi(0.0)
    slope = 3 * math.sinh(-2.4)  # phi'(0)
    prev = None
    for K in (2, 3, 5, 8):
        h, f, calls = oracle_mod.ls_par(phi, f0, slope, 0.1, K=K, g0=1)
        assert len(calls) == K + 1
        assert f < f0
        if prev is not None:
            assert f <= prev + 1e-15
        prev = f
    from scipy.optimize import minimize_scalar
    hmin = minimize_scalar(phi, bounds=(0, 2), method="bounded", options={"xatol": 1e-10}).x
    assert h == pytest.approx(hmin, abs=1e-4)


def test_ls_par_degenerate_concave(oracle_mod):
    # phi = -h^2, slope 0: G0 curvature -1 -> h2 = k+ h1; 3-point fit concave
    # -> h3 = k+ * (best h) = 4 h0 (reading of the degenerate case).
    phi = lambda h: -h * h
    h, f, calls = oracle_mod.ls_par(phi, 0.0, 0.0, 0.1, K=2, g0=1)
    assert calls == pytest.approx([0.1, 0.2, 0.4])
    assert h == pytest.approx(0.4) and f == pytest.approx(-0.16)


def test_ls_par_failure_returns_zero(oracle_mod):
    phi = lambda h: abs(h)  # no descent anywhere
    h, f, calls = oracle_mod.ls_par(phi, 0.0, -1.0, 0.1, K=2, g0=1)
    assert h == 0.0 and f == 0.0


def test_ls_h_expands_on_decrease(oracle_mod):
    # strictly decreasing: f(h0) < f* -> one try at k+ h0, which is better
    h, f, calls = oracle_mod.ls_h(lambda h: -h, 0.0, 0.1)
    assert calls == [0.1, 0.2] and h == 0.2 and f == -0.2


def test_ls_h_keeps_h0_when_expansion_worse(oracle_mod):
    phi = lambda h: (h - 0.12) ** 2 - 0.0144  # phi(0) = 0
    h, f, calls = oracle_mod.ls_h(phi, 0.0, 0.1)
    assert calls == [0.1, 0.2] and h == 0.1


def test_ls_h_shrinks_until_relaxing(oracle_mod):
    # f(h) = (h - 0.001)^2 - 1e-6 from h0 = 0.1: first h = 0.1 * 0.5^j with f < 0
    phi = lambda h: (h - 0.001) ** 2 - 1e-6
    h, f, calls = oracle_mod.ls_h(phi, 0.0, 0.1)
    j = next(j for j in range(1, 60) if phi(0.1 * 0.5 ** j) <= 0.0)
    assert h == pytest.approx(0.1 * 0.5 ** j, rel=1e-15)
    assert len(calls) == j + 1


def test_ls_h_failure_when_increasing(oracle_mod):
    h, f, calls = oracle_mod.ls_h(lambda h: h, 0.0, 0.1, eps_h=1e-10)
    # evaluations at 0.1, 0.05, ... until 0.1 * 0.5^j <= 1e-10 stops the loop
    jstop = next(j for j in range(1, 100) if 0.1 * 0.5 ** j <= 1e-10)
    assert h == 0.0 and f == 0.0
    assert len(calls) == jstop  # h0 plus every shrunk step above eps_h


def test_ls_h_accepts_equal_value(oracle_mod):
    # the loop test is strict (f > f*): f == f* ends the search (Alg. 5)
    h, f, calls = oracle_mod.ls_h(lambda h: 0.0 if h < 0.06 else 1.0, 0.0, 0.1)
    assert h == 0.05 and f == 0.0


# ------------------------------ quadratic pins ------------------------------

def spd(n, cond, seed):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = np.geomspace(1.0, cond, n)
    return (q * lam) @ q.T, rng.normal(size=n), lam


def quad_fg(A, b):
    def fg(x, want):
        Ax = A @ x
        return 0.5 * x @ Ax - b @ x, (Ax - b if want else None)
    return fg


def test_gd_kantorovich_rate(oracle_mod):
    # steepest descent with exact line search (LS_PAR is exact on a
    # quadratic): f_{k+1} - f* <= ((k-1)/(k+1))^2 (f_k - f*) (Eq. 3-type bound)
    A, b, lam = spd(10, 30.0, 1)
    xs = np.linalg.solve(A, b)
    fstar = 0.5 * xs @ A @ xs - b @ xs
    x0 = np.zeros(10)
    xo, r = oracle_mod.minimize_fn(quad_fg(A, b), x0, method=oracle_mod.GD, gtol_inf=1e-5,
                                   max_iter=400, ls_par_g0=1)
    tr = oracle_mod.trace()["f"]
    f0 = quad_fg(A, b)(x0, False)[0]
    seq = np.concatenate([[f0], tr]) - fstar
    kappa = lam[-1] / lam[0]
    bound = ((kappa - 1) / (kappa + 1)) ** 2
    ok = seq[:-1] > 1e-12
    ratios = seq[1:][ok] / seq[:-1][ok]
    assert ratios.max() <= bound + 1e-9
    assert r["status_name"] == "ok"


@pytest.mark.parametrize("variant", range(7))
def test_cg_finite_termination(oracle_mod, variant):
    # CG with exact searches terminates in <= n steps on an SPD quadratic
    # (Section 4, Eq. 7 with N = n); every beta variant coincides there.
    n = 8
    A, b, _ = spd(n, 50.0, 2)
    xo, r = oracle_mod.minimize_fn(quad_fg(A, b), np.zeros(n), method=oracle_mod.CG,
                                   cg_variant=variant, gtol_inf=1e-8, max_iter=50,
                                   cg_restart_every=1000)
    assert r["status_name"] == "ok"
    assert r["iterations"] <= n + 1
    assert np.abs(xo - np.linalg.solve(A, b)).max() < 1e-6


def test_lbfgs_finite_termination(oracle_mod):
    n = 8
    A, b, _ = spd(n, 50.0, 3)
    xo, r = oracle_mod.minimize_fn(quad_fg(A, b), np.zeros(n), method=oracle_mod.LBFGS,
                                   lbfgs_m=10, gtol_inf=1e-8, max_iter=50)
    assert r["status_name"] == "ok" and r["iterations"] <= n + 1


def bfgs_matrix(S, Y, H0):
    # explicit inverse-Hessian BFGS updates H+ = V^T H V + rho s s^T,
    # V = I - rho y s^T (Nocedal & Wright, Eq. 6.17), oldest pair first
    H = H0.copy()
    n = H.shape[0]
    for s, y in zip(S, Y):
        rho = 1.0 / (s @ y)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


@pytest.mark.parametrize("count", [1, 3, 6])
@pytest.mark.parametrize("diag", [False, True])
def test_lbfgs_two_loop_equals_bfgs_matrix(oracle_mod, count, diag):
    rng = np.random.default_rng(count)
    n = 12
    A, _, _ = spd(n, 20.0, 9)
    S = rng.normal(size=(count, n))
    Y = S @ A.T  # curvature pairs of a quadratic: <s, y> > 0
    g = rng.normal(size=n)
    d = rng.uniform(0.5, 2.0, size=n) if diag else np.ones(n)
    gamma = S[-1] @ Y[-1] / (Y[-1] @ Y[-1])
    H = bfgs_matrix(S, Y, gamma * np.diag(d))
    r = oracle_mod.lbfgs_direction(g, S, Y, d if diag else None)
    assert np.allclose(r, -H @ g, rtol=1e-10, atol=1e-12)


def test_fgm_theta_recurrence(oracle_mod):
    # theta_k solves theta^2 = (1 - theta) theta_{k-1}^2 (Alg. 1's update is the
    # positive root), theta_{-1} = 1; the literal method never resets theta;
    # beta_k in [0, 1)
    A, b, _ = spd(10, 100.0, 4)
    xo, r = oracle_mod.minimize_fn(quad_fg(A, b), np.zeros(10), method=oracle_mod.FGM,
                                   gtol_inf=1e-6, max_iter=500)
    tr = oracle_mod.trace()
    th = np.concatenate([[1.0], tr["theta"]])
    assert len(th) > 5
    assert np.all(np.diff(th) < 0.0)
    assert np.allclose(th[1:] ** 2, (1 - th[1:]) * th[:-1] ** 2, rtol=1e-12, atol=0.0)
    assert np.all(tr["beta"] >= 0.0) and np.all(tr["beta"] < 1.0)
    # with LS_H the literal method need not converge here; it returns its best point
    assert r["energy"] == pytest.approx(min(0.0, tr["f"].min()), rel=1e-12)
    assert 0.5 * xo @ A @ xo - b @ xo == pytest.approx(r["energy"], rel=1e-12)


def fista_form(A, b, L, x0, steps):
    """Nesterov's accelerated gradient in the t-form of Beck and Teboulle
    (SIAM J. Imaging Sci. 2009, FISTA with an identity proximal map):
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, y = x_k + (t_{k-1} - 1)/t_k (x_k - x_{k-1}),
    x_{k+1} = y - grad f(y) / L.  Started from t = 1 then t = (1 + sqrt 5)/2,
    the start of Nesterov's constant-step scheme (2.2.19) with
    alpha_0 = (sqrt 5 - 1)/2 = 1/t.  Returns the iterates x_1 .. x_steps."""
    x, xp = x0.copy(), x0.copy()
    t_prev, t = 1.0, 0.5 * (1.0 + np.sqrt(5.0))
    out = []
    for _ in range(steps):
        y = x + (t_prev - 1.0) / t * (x - xp)
        xp, x = x, y - (A @ y - b) / L
        t_prev, t = t, 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        out.append(x.copy())
    return out


@pytest.mark.parametrize("N", [1, 2, 7, 40])
def test_fgm_fixed_step_equals_fista_form(oracle_mod, N):
    # Algorithm 1 with the fixed step 1/L in place of the line search is
    # Nesterov's method; its theta / beta recurrence (beta_k and the
    # extrapolation w^k = x^k + beta_k (x^k - x^{k-1})) must give the same
    # iterates as the independent t-form above.  A dropped term of beta, a
    # theta_k written for theta_{k-1} or a sign slip in w breaks this.
    A, b, lam = spd(12, 200.0, 5)
    L = lam[-1]
    x0 = np.random.default_rng(2).normal(size=12)
    xs = fista_form(A, b, L, x0, N)
    fs = np.array([0.5 * x @ A @ x - b @ x for x in xs])
    xo, r = oracle_mod.minimize_fn(quad_fg(A, b), x0, method=oracle_mod.FGM, gtol_inf=1e-14,
                                   max_iter=N, fgm_step=1.0 / L)
    assert r["iterations"] == N
    tr = oracle_mod.trace()
    assert np.allclose(tr["f"], fs, rtol=1e-12, atol=1e-12)
    # the method returns its best point x_* (Algorithm 1)
    f0 = 0.5 * x0 @ A @ x0 - b @ x0
    best = x0 if f0 <= fs.min() else xs[int(np.argmin(fs))]
    assert np.abs(xo - best).max() <= 1e-11 * (1.0 + np.abs(best).max())


@pytest.mark.parametrize("seed", range(4))
def test_fgm_rate_on_convex_quadratics(oracle_mod, seed):
    # Nesterov (Introductory Lectures 2004, Theorem 2.2.3) for scheme (2.2.19)
    # with mu = 0 and alpha_0 = (sqrt 5 - 1)/2, i.e. gamma_0 = L:
    #   f(x_k) - f* <= 4 (f(x_0) - f* + L R^2 / 2) / (k + 2)^2
    n = 30
    A, b, lam = spd(n, 1000.0, seed)
    L = lam[-1]
    xs = np.linalg.solve(A, b)
    fstar = 0.5 * xs @ A @ xs - b @ xs
    x0 = np.zeros(n)
    oracle_mod.minimize_fn(quad_fg(A, b), x0, method=oracle_mod.FGM, gtol_inf=1e-9,
                           max_iter=2000, fgm_step=1.0 / L)
    f = oracle_mod.trace()["f"] - fstar
    k = np.arange(1, len(f) + 1)
    f0 = 0.5 * x0 @ A @ x0 - b @ x0 - fstar
    assert len(f) > 500
    assert np.all(f <= 4.0 * (f0 + 0.5 * L * np.sum((x0 - xs) ** 2)) / (k + 2) ** 2 * (1 + 1e-9))


def test_fgm_literal_keeps_best_point_and_restart_option(oracle_mod):
    # Section 5.1: FGM is non-monotone (f(x^{k+1}) > f(x^k) happens) and
    # returns the best point x_*.  On the clashing force-field start the
    # literal method reaches its best point early and then wanders with
    # beta -> 1; the optional function-value restart (not in Algorithm 1)
    # resets theta and converges.
    s = synth.make_system(40, 21)
    e0 = oracle_mod.energy(s, s.x)
    xo, r = oracle_mod.minimize(s, s.x, method=oracle_mod.FGM, max_iter=400)
    tr = oracle_mod.trace()
    assert r["status_name"] == "max_iter" and len(tr["f"]) == 400
    assert np.any(np.diff(tr["f"]) > 0.0)  # non-monotone
    assert np.all(np.diff(np.concatenate([[1.0], tr["theta"]])) < 0.0)  # never reset
    best = min(e0, tr["f"].min())
    e1, g1 = oracle_mod.energy_grad(s, xo)
    assert r["energy"] == pytest.approx(best, rel=1e-12)
    assert e1 == pytest.approx(best, rel=1e-12)
    assert np.abs(g1).max() == pytest.approx(r["grad_inf"], rel=1e-12)
    xo, r = oracle_mod.minimize(s, s.x, method=oracle_mod.FGM, max_iter=20000, fgm_restart=1)
    th = oracle_mod.trace()["theta"]
    assert np.any(np.diff(th) > 0.0)  # restarts happened
    assert r["status_name"] == "ok" and r["energy"] < best


def test_ogm_first_step_is_cauchy_step(oracle_mod):
    # with t_0 = 1 the first OGM step has y = x^0 and d = (1 + 1/t_1) grad f(x^0),
    # i.e. steepest descent with an exact search (LS_PAR is exact on a
    # quadratic): the Cauchy point x^0 - (g.g / g.Ag) g
    A, b, _ = spd(10, 50.0, 3)
    x0 = np.zeros(10)
    g = A @ x0 - b
    x1 = x0 - (g @ g) / (g @ A @ g) * g
    xo, r = oracle_mod.minimize_fn(quad_fg(A, b), x0, method=oracle_mod.OGM, gtol_inf=1e-12,
                                   max_iter=1)
    assert r["iterations"] == 1
    assert np.abs(xo - x1).max() < 1e-12 * (1 + np.abs(x1).max())


@pytest.mark.parametrize("N", [1, 2, 7, 40])
def test_ogm_fixed_step_equals_kim_fessler(oracle_mod, N):
    # Eq. 11 with the fixed step 1/L is Drori and Teboulle's efficient form of
    # the optimized gradient method; Kim and Fessler (Math. Prog. 2016) give
    # the same iterates in momentum form:
    #   y_{k+1} = x_k - grad f(x_k) / L,
    #   x_{k+1} = y_{k+1} + (t_k - 1)/t_{k+1} (y_{k+1} - y_k)
    #                     + t_k/t_{k+1} (y_{k+1} - x_k),   y_0 = x_0, t_0 = 1
    A, b, lam = spd(12, 200.0, 5)
    L = lam[-1]
    x0 = np.random.default_rng(1).normal(size=12)
    x, yp, t = x0.copy(), x0.copy(), 1.0
    for _ in range(N):
        y = x - (A @ x - b) / L
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        x = y + (t - 1.0) / tn * (y - yp) + t / tn * (y - x)
        yp, t = y, tn
    xo, r = oracle_mod.minimize_fn(quad_fg(A, b), x0, method=oracle_mod.OGM, gtol_inf=1e-14,
                                   max_iter=N, ogm_step=1.0 / L)
    assert r["iterations"] == N
    assert np.abs(xo - x).max() <= 1e-11 * (1.0 + np.abs(x).max())


@pytest.mark.parametrize("seed", range(4))
def test_ogm_rate_on_convex_quadratics(oracle_mod, seed):
    # Section 4, Eq. 12 (and the sentence after Eq. 13: the same bound holds
    # with the step chosen by a line search): f(x^N) - f* <= L R^2 / N^2
    n = 30
    A, b, lam = spd(n, 1000.0, seed)
    xs = np.linalg.solve(A, b)
    fstar = 0.5 * xs @ A @ xs - b @ xs
    x0 = np.zeros(n)
    xo, r = oracle_mod.minimize_fn(quad_fg(A, b), x0, method=oracle_mod.OGM, gtol_inf=1e-7,
                                   max_iter=1500)
    f = oracle_mod.trace()["f"] - fstar
    N = np.arange(1, len(f) + 1)
    assert len(f) > 100
    assert np.all(f <= lam[-1] * np.sum((x0 - xs) ** 2) / N ** 2 * (1 + 1e-9))
    # t_{k+1} = (1 + sqrt(4 t_k^2 + 1)) / 2 from t_0 = 1
    t = oracle_mod.trace()["theta"]
    assert t[0] == pytest.approx((1 + np.sqrt(5.0)) / 2, rel=1e-15)
    assert np.allclose(t[1:], (1 + np.sqrt(4 * t[:-1] ** 2 + 1)) / 2, rtol=1e-14)


# ------------------------------ force field ------------------------------

@pytest.mark.parametrize("method", ["GD", "FGM", "CG", "LBFGS"])
def test_force_field_minimizers_converge(oracle_mod, method):
    # (FGM with the optional momentum restart: the literal Algorithm 1 does
    # not converge from this start, see the test above)
    s = synth.make_system(40, 21)
    e0 = oracle_mod.energy(s, s.x)
    xo, r = oracle_mod.minimize(s, s.x, method=getattr(oracle_mod, method), max_iter=20000,
                                fgm_restart=int(method == "FGM"))
    assert r["status_name"] == "ok", r
    assert r["grad_inf"] < 0.1
    e1, g1 = oracle_mod.energy_grad(s, xo)
    assert r["energy"] == pytest.approx(e1, rel=1e-12)
    assert np.abs(g1).max() == pytest.approx(r["grad_inf"], rel=1e-12)
    assert e1 < e0


def test_force_field_ogm(oracle_mod):
    # the literal OGM is slow on this non-convex landscape (Section 4's
    # remark that CG-type methods win in practice) but must lower the
    # energy and report the returned point
    s = synth.make_system(40, 21)
    e0 = oracle_mod.energy(s, s.x)
    xo, r = oracle_mod.minimize(s, s.x, method=oracle_mod.OGM, max_iter=2000)
    assert r["status_name"] in ("ok", "max_iter"), r
    e1, g1 = oracle_mod.energy_grad(s, xo)
    assert r["energy"] == pytest.approx(e1, rel=1e-12)
    assert np.abs(g1).max() == pytest.approx(r["grad_inf"], rel=1e-12)
    assert e1 < 1e-3 * e0


def parab_brute_force(oracle_mod, s, x, moves, seed, delta):
    # the gradient-free move (Section 3) with every trial energy taken as a
    # full-energy difference (brute force)
    x = x.copy()
    n = x.shape[0]
    for t in range(moves):
        i = oracle_mod.pick_atom(seed, t, n)
        base = oracle_mod.energy(s, x)
        pts = [x[i].copy()]
        for a in range(3):
            for sgn in (1, -1):
                p = x[i].copy(); p[a] += sgn * delta; pts.append(p)

        def de(p):
            y = x.copy(); y[i] = p
            return oracle_mod.energy(s, y) - base

        f = [de(p) for p in pts]
        v = x[i].copy()
        for a in range(3):
            fp, fm = f[1 + 2 * a], f[2 + 2 * a]
            curv = fm - 2 * f[0] + fp
            v[a] += delta * (fm - fp) / (2 * curv) if curv > 0 else 0.0
        pts.append(v); f.append(de(v))
        x[i] = pts[int(np.argmin(f))]
    return x


def test_parab_matches_brute_force(oracle_mod):
    s = synth.make_system(8, 31)
    moves = 40
    xo, r = oracle_mod.minimize(s, s.x, method=oracle_mod.GRADFREE, max_iter=moves,
                                gtol_inf=1e-12, seed=77, gradfree_delta=0.05)
    xb = parab_brute_force(oracle_mod, s, s.x, moves, 77, 0.05)
    assert r["iterations"] == moves and r["status_name"] == "max_iter"
    assert np.abs(xo - xb).max() < 1e-9
    assert oracle_mod.energy(s, xo) <= oracle_mod.energy(s, s.x)


def test_parab_energy_never_increases(oracle_mod):
    s = synth.make_system(30, 32)
    e = oracle_mod.energy(s, s.x)
    x = s.x.copy()
    for chunk in range(5):
        x, r = oracle_mod.minimize(s, x, method=oracle_mod.GRADFREE, max_iter=30,
                                   gtol_inf=1e-12, seed=100 + chunk)
        e2 = oracle_mod.energy(s, x)
        assert e2 <= e + 1e-9 * abs(e)
        e = e2
