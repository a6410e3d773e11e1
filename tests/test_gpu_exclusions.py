"""GPU parity of the exclusion variant (bonded and angle-end pairs excluded,
dihedral-end pairs scaled by scale14; a force-field option outside the
paper) with the FP64 oracle, through the C ABI.  The GPU keeps its
all-pairs sweep and adds FP64 correction terms of weight s_ij - 1, so the
bars are those of the plain energy tests (FP64) plus the cancellation of
the excluded terms: E within 2e-11 of sum|terms| and the gradient within
1e-9 of the largest force, both taken over every term the sweep evaluates
(the all-pairs sums, which include the excluded clashes).

MIXED objects: an FP32 correction could not cancel the sweep's rounding of
the excluded bonded-neighbour clashes (up to 1e10 kcal/mol at a jittered
start), so the FP32 sweeps scale the listed pairs inside their sums (the
tiles holding scaled partners take a masked sweep).  The MIXED bars are then
those of the plain MIXED path relative to the variant's own terms: E within
1e-5 of sum|terms| plus the FP32 position-rounding bound, the gradient
within 1e-4 of the largest force; difference trials within the same bar of
sum |term differences|."""
import dataclasses

import numpy as np
import pytest

from paper_1810_03358_gb300 import synth
from tests.gpu_util import mixed_position_bound, need_gpu, split, to_dev
from tests.test_gpu_minimize import ensemble_parity, prefix_parity, PREFIX, run_gpu

pytestmark = pytest.mark.gpu

TOL = {0: dict(e=2e-11, g=1e-9)}


@pytest.fixture(scope="module")
def ff():
    return need_gpu()


def excl(s, scale14=0.5):
    return dataclasses.replace(s, exclusions=1, scale14=scale14)


def check(ffmin, oracle_mod, systems, prec, xs=None):
    xs = xs or [s.x for s in systems]
    S = ffmin.System(systems, prec)
    x = to_dev(xs)
    e, g = S.energy_grad(x)
    e_only = S.energy(x)
    g = split(g.cpu().numpy(), systems)
    S.close()
    for b, s in enumerate(systems):
        d, st, go = oracle_mod.energy_terms(s, xs[b], grad=True)
        assert st == 0
        # the sweep still evaluates the excluded pairs (clashes of bonded
        # neighbours, up to 1e10 kcal/mol at a jittered start) and the
        # corrections cancel them: the rounding bars are those of the plain
        # path relative to every term evaluated, i.e. the all-pairs sums
        d0, _, g0 = oracle_mod.energy_terms(dataclasses.replace(s, exclusions=0), xs[b], grad=True)
        e_tol = TOL[prec]["e"] * max(d["sum_abs"], d0["sum_abs"])
        g_tol = TOL[prec]["g"] * max(np.abs(go).max(), np.abs(g0).max())
        assert abs(e[b] - d["total"]) <= e_tol, (b, e[b], d["total"])
        # and the stated bars against the variant's own terms
        assert abs(e[b] - d["total"]) <= 1e-6 * d["sum_abs"]
        assert np.abs(g[b] - go).max() <= 1e-4 * np.abs(go).max()
        assert abs(e_only[b] - e[b]) <= e_tol
        assert np.abs(g[b] - go).max() <= g_tol, b


@pytest.mark.parametrize("n", [3, 4, 64, 129, 300])
def test_energy_gradient(ff, oracle_mod, n):
    check(ff, oracle_mod, [excl(synth.make_system(n, 600 + n))], 0)


def check_mixed(ffmin, oracle_mod, systems, xs=None, tuning=None):
    xs = xs or [s.x for s in systems]
    S = ffmin.System(systems, 1)
    if tuning is not None:
        S.set_tuning(*tuning)
    x = to_dev(xs)
    e, g = S.energy_grad(x)
    e_only = S.energy(x)
    g = split(g.cpu().numpy(), systems)
    S.close()
    for b, s in enumerate(systems):
        d, st, go = oracle_mod.energy_terms(s, xs[b], grad=True)
        assert st == 0
        bar = 1e-5 + mixed_position_bound(xs[b])
        assert abs(e[b] - d["total"]) <= bar * d["sum_abs"], (b, e[b], d["total"], bar)
        assert abs(e_only[b] - d["total"]) <= bar * d["sum_abs"], (b, e_only[b], d["total"])
        # near a minimum the force scale is the stopping tolerance: the bar is
        # then 2 % of it in absolute terms (as for the plain MIXED path)
        assert np.abs(g[b] - go).max() <= max(1e-4 * np.abs(go).max(), 0.02 * 0.1), b


@pytest.mark.parametrize("n", [3, 4, 64, 129, 300, 1000])
def test_mixed_energy_gradient(ff, oracle_mod, n):
    check_mixed(ff, oracle_mod, [excl(synth.make_system(n, 600 + n))])


@pytest.mark.parametrize("ipt", [1, 2])
def test_mixed_tile_shapes(ff, oracle_mod, ipt):
    # the masked FP32 sweeps in both tile shapes (one or two i-atoms per
    # thread), a partial tile and a several-tile system in one batch
    systems = [excl(synth.make_system(n, 640 + n)) for n in (70, 400, 1000)]
    check_mixed(ff, oracle_mod, systems, tuning=(10, ipt))


def test_mixed_batch_and_minimized_geometry(ff, oracle_mod):
    # a batch of 10 (per-system reductions) mixing systems with and without
    # exclusions, and a geometry near a minimum of the variant
    systems = [excl(synth.make_system(40 + 37 * k, 620 + k), 0.5) if k % 3 else synth.make_system(40 + 37 * k, 620 + k)
               for k in range(10)]
    check_mixed(ff, oracle_mod, systems)
    s = excl(synth.make_system(120, 613))
    xo, ro = oracle_mod.minimize(s, s.x, method=3)
    check_mixed(ff, oracle_mod, [s], [xo])


def test_mixed_difference_trials(ff, oracle_mod):
    # line-search trials of the variant in MIXED precision against the
    # oracle's term-by-term differences (excluded pairs contribute nothing,
    # 1-4 pairs their scaled difference)
    s = excl(synth.make_system(500, 631))
    _, g = oracle_mod.energy_grad(s, s.x)
    r = -g.reshape(-1) / np.linalg.norm(g)
    S = ff.System([s], 1)
    x, rd = to_dev([s.x]), to_dev([r])
    bar = 1e-5 + mixed_position_bound(s.x)
    for h in (1e-3, 1e-2, 0.1):
        de = S.energy_delta(x, rd, h)[0]
        dref, aref, st = oracle_mod.energy_delta(s, s.x, s.x + h * r.reshape(-1, 3))
        assert st == 0
        assert abs(de - dref) <= bar * aref, (h, de, dref)
    S.close()


def test_mixed_minimization(ff, oracle_mod):
    # MIXED L-BFGS of the variant: certified by the FP64 phase, held to the
    # fixed oracle ensemble one-sided; the MIXED gradient-free search of the
    # variant is refused (its FP32 rows do not mask the excluded pairs)
    s = excl(synth.make_system(90, 632))
    kw = dict(method=3, max_iter=100000)
    xg, rg, _ = run_gpu(ff, [s], 1, **kw)
    ensemble_parity(oracle_mod, s, xg[0], rg[0], kw, mixed=True)
    S = ff.System([s], 1)
    with pytest.raises(ff.FfminError) as ei:
        S.minimize(to_dev([s.x]), method=4, max_iter=10)
    assert ei.value.status == ff.FFMIN_ERR_INVALID_ARG
    S.close()


@pytest.mark.parametrize("scale14", [0.0, 1.0 / 1.2, 1.0])
def test_scale14_values_and_mixed_batch(ff, oracle_mod, scale14):
    # a batch mixing systems with and without exclusions
    systems = [excl(synth.make_system(70, 610), scale14), synth.make_system(50, 611),
               excl(synth.make_system(140, 612), scale14)]
    check(ff, oracle_mod, systems, 0)


def test_minimized_geometry_fp64(ff, oracle_mod):
    s = excl(synth.make_system(120, 613))
    xo, ro = oracle_mod.minimize(s, s.x, method=3)
    assert ro["status_name"] == "ok"
    check(ff, oracle_mod, [s], 0, [xo])


def test_invalid_scale14_rejected(ff):
    s = dataclasses.replace(synth.make_system(10, 614), exclusions=1, scale14=float("nan"))
    with pytest.raises(ff.FfminError):
        ff.System([s], 0)


def test_lbfgs_prefix_and_full_run(ff, oracle_mod):
    s = excl(synth.make_system(80, 615))
    kw = dict(method=3, max_iter=PREFIX)
    xg, rg, _ = run_gpu(ff, [s], 0, **kw)
    prefix_parity(oracle_mod, s, xg[0], rg[0], kw)
    kw = dict(method=3, max_iter=100000)
    xg, rg, _ = run_gpu(ff, [s], 0, **kw)
    ensemble_parity(oracle_mod, s, xg[0], rg[0], kw)


def test_gradient_free_moves(ff, oracle_mod):
    # the row energies of the moved atom include its exclusion corrections
    s = excl(synth.make_system(90, 617))
    kw = dict(method=4, max_iter=400, gtol_inf=1e-9, seed=77, gradfree_delta=0.05)
    S = ff.System([s], 0)
    x = to_dev([s.x])
    r = S.minimize(x, **kw)[0]
    S.close()
    xo, ro = oracle_mod.minimize(s, s.x, **kw)
    assert r["iterations"] == ro["iterations"] == 400
    # same decision at every move (another choice moves an atom by ~delta);
    # the parabola vertices inherit the rounding of the row energies, which
    # here includes the cancelled clashes of the excluded neighbours
    # (~1e-16 of 1e10 kcal/mol), hence 1e-6 A rather than the 1e-9 A of
    # the plain force field
    assert np.abs(x.cpu().numpy().reshape(-1, 3) - xo).max() < 1e-6
