"""Parity of the device-resident minimizers (Algorithms 1-6, Eq. 4) with the
FP64 oracle, through the C ABI.

Two bars (FP64 path):

1. Prefix parity.  Both sides take the same decisions on energies that
   differ only in summation order, so a capped run
   must reproduce the oracle step for step: same iteration and evaluation
   counts, same stop reason, final energy within 1e-8 relative and the
   returned point within 1e-6 A.  The cap is 60 accepted steps: measured
   differences grow about 1.14x per step from rounding level (1e-16) in
   most cases, i.e. ~1e-12 at 60 steps.  Where the oracle's own capped run
   is more sensitive (CG with LS_H on the 50-atom system moves by 3e-7 in
   energy when its start moves by 1e-15 A), the energy and coordinate bars
   become 10x that measured self-sensitivity.

2. Full runs.  After a few hundred steps the two trajectories, equal up to
   rounding, separate (the landscape is rugged: measured agreement 1e-12 at
   300 steps, 1e-7 at 1000) and end in neighbouring minima.  The oracle's
   final energy is itself only defined up to that chaos, so a full run is
   compared with an ensemble of oracle runs from starts perturbed by
   1e-12 A: the GPU's final energy must lie within 0.01 % of the ensemble's
   range (or below it by at most the ensemble's own spread), or else within
   0.01 % of some further oracle run from a start perturbed by 1e-12 to
   1e-6 A (the GPU run reached a basin those members missed); its stop must
   be valid (converged with the oracle's own gradient of the returned point
   below the tolerance), and the reported energy must be the energy of the
   returned point.
"""
import numpy as np
import pytest

from paper_1810_03358_gb300 import synth
from tests.gpu_util import _oracle_minimize, need_gpu, oracle_map, split, to_dev

pytestmark = pytest.mark.gpu

REL_E = 1e-4  # 0.01 %
# capped prefix: measured divergence grows ~1.14x per step from 1e-16, so 60
# steps keep the two trajectories equal to ~1e-12
PREFIX = 60
# Algorithm 1 as printed (FGM without restart) reaches its best point within
# ~30 steps on these clashing starts and then runs with beta -> 1, which
# amplifies rounding differences far faster: its line searches' evaluation
# counts become rounding-decided (the oracle's own runs from starts 1e-15 ..
# 1e-13 A apart differ by 1 or 2).  Its exact-count prefix is 25 steps; at
# 60 steps its returned best point is compared (unique and robust).
PREFIX_FGM = 25


def fgm_literal(kw):
    return kw.get("method") == 1 and not kw.get("fgm_restart", 0)


def prefix_or_best(oracle_mod, s, ff, systems_prec, kw):
    """Prefix parity; for literal FGM the 25-step prefix plus the 60-step
    best point (energy within 1e-8, coordinates within 1e-6 A)."""
    if not fgm_literal(kw):
        xg, rg, _ = run_gpu(ff, [s], systems_prec, **kw)
        prefix_parity(oracle_mod, s, xg[0], rg[0], kw)
        return
    k25 = dict(kw, max_iter=PREFIX_FGM)
    xg, rg, _ = run_gpu(ff, [s], systems_prec, **k25)
    prefix_parity(oracle_mod, s, xg[0], rg[0], k25)
    xg, rg, _ = run_gpu(ff, [s], systems_prec, **kw)
    xo, ro = oracle_mod.minimize(s, s.x, **kw)
    assert rg[0]["iterations"] == ro["iterations"] and rg[0]["status_name"] == ro["status_name"]
    assert abs(rg[0]["energy"] - ro["energy"]) <= 1e-8 * abs(ro["energy"]), (rg[0], ro)
    assert np.abs(xg[0] - xo).max() <= 1e-6
STATUS = {"ok": "ok", "linesearch": "linesearch", "max_iter": "max_iter", "nonfinite": "nonfinite"}


@pytest.fixture(scope="module")
def ff():
    return need_gpu()


def run_gpu(ffmin, systems, prec, **opts):
    S = ffmin.System(systems, prec)
    x = to_dev([s.x for s in systems])
    res = S.minimize(x, **opts)
    xs = split(x.cpu().numpy(), systems)
    stats = S.last_stats()
    S.close()
    return xs, res, stats


COUNTS = ("iterations", "energy_evals", "grad_evals", "ls_failures")


def oracle_sensitivity(oracle_mod, s, xo, ro, kw, eps=(1e-15, 1e-14, 1e-13)):
    """How far the oracle's own capped run moves when its start moves by a
    rounding-scale amount: one member per eps (A).  The GPU's rounding
    differs from the oracle's in every evaluation of the run, not only at
    the start: about sqrt(60) evaluations' worth of ~u |x| = 4e-15 A, i.e.
    up to ~3e-14 A, which the members bracket.  Returns (max relative
    energy change, max coordinate change, the members' count tuples)."""
    de, dx, counts = 0.0, 0.0, []
    for k, e in enumerate(eps, start=1):
        x0 = s.x + e * np.random.default_rng(k).normal(size=s.x.shape)
        x1, r1 = oracle_mod.minimize(s, x0, **kw)
        de = max(de, abs(r1["energy"] - ro["energy"]) / abs(ro["energy"]))
        dx = max(dx, float(np.abs(x1 - xo).max()))
        counts.append(tuple(r1[c] for c in COUNTS))
    return de, dx, counts


def prefix_parity(oracle_mod, s, xg, rg, kw, ref=None):
    xo, ro = ref if ref is not None else oracle_mod.minimize(s, s.x, **kw)
    assert rg["status_name"] == STATUS[ro["status_name"]], (rg, ro)
    same_counts = all(rg[k] == ro[k] for k in COUNTS)
    de = abs(rg["energy"] - ro["energy"]) / abs(ro["energy"])
    dx = float(np.abs(xg - xo).max())
    if same_counts and de <= 1e-8 and dx <= 1e-6:
        return
    # some capped runs are chaotic already within the prefix: the oracle's
    # own run, restarted a rounding-scale distance away, moves by a
    # comparable amount.  The GPU run (different summation order, i.e.
    # rounding-level differences in every evaluation) must then stay within
    # 10x that self-sensitivity; its counts may differ from the oracle's only
    # where the oracle's own counts flip under such a perturbation (a
    # line-search comparison decided by rounding), and must then equal a
    # member's.
    se, sx, counts = oracle_sensitivity(oracle_mod, s, xo, ro, kw)
    if not same_counts:
        assert tuple(rg[k] for k in COUNTS) in counts, (rg, ro, counts)
    assert de <= max(1e-8, 10.0 * se), (de, se, rg, ro)
    assert dx <= max(1e-6, 10.0 * sx), (dx, sx)


# the fixed oracle ensemble of a full run: the start itself and starts
# perturbed by 1e-12 .. 1e-6 A (seeds 1 .. 6).  1e-12 A is the rounding
# scale of the FP64 path's differences; 1e-6 A that of FP32 coordinates
# (u |x| at 20 A), the perturbation a MIXED trajectory carries
ENSEMBLE_EPS = (0.0, 1e-12, 1e-12, 1e-10, 1e-8, 1e-6, 1e-6)


def oracle_ensemble(s, kw):
    starts = [s.x if e == 0.0 else s.x + e * np.random.default_rng(k).normal(size=s.x.shape)
              for k, e in enumerate(ENSEMBLE_EPS)]
    n = len(starts)
    out = oracle_map(_oracle_minimize, [s] * n, starts, [kw] * n)
    return [r["energy"] for _, r in out if r["status_name"] == "ok"]


def ensemble_parity(oracle_mod, s, xg, rg, kw, energies=None, mixed=False):
    """A full run against the fixed oracle ensemble: its final energy lies
    within 0.01 % of the members' range (or below it by at most the range
    itself), or within 0.01 % of one member; it is a valid stop (the
    oracle's gradient of the returned point below the tolerance) and reports
    that point's energy.  A MIXED run (FP32 trials take other decisions
    from the first steps on, so it ends in whichever basin its own
    trajectory reaches) is held one-sided: no higher than the highest member
    by more than max(0.01 %, the members' own spread), the scale at which
    runs perturbed by rounding already choose different basins (measured
    spreads 6.6e-4 to 1.5e-3); a deeper minimum than the members' is a valid
    result (measured: up to 0.23 % below).  Prints which criterion held."""
    if energies is None:
        energies = oracle_ensemble(s, kw)
    assert energies, "the oracle itself did not converge"
    lo, hi = min(energies), max(energies)
    tol = REL_E * max(abs(lo), abs(hi))
    e = rg["energy"]
    in_range = lo - max(tol, hi - lo) <= e <= hi + tol
    near = any(abs(m - e) <= REL_E * abs(e) for m in energies)
    below = mixed and e <= hi + max(tol, hi - lo)
    print(f"ensemble ({len(energies)} members, spread {(hi - lo) / abs(lo):.1e}): "
          f"{'range' if in_range else ('member' if near else ('spread' if below else 'miss'))}, "
          f"gpu {e:.10g} ({(e - lo) / abs(lo):+.1e} from the lowest member)")
    assert in_range or near or below, (e, energies)
    assert rg["status_name"] == "ok", rg
    e_ret, g_ret = oracle_mod.energy_grad(s, xg)
    assert abs(e_ret - e) <= 1e-9 * max(abs(e_ret), 1.0)
    assert np.abs(g_ret).max() < kw.get("gtol_inf", 0.1) * (1 + 1e-6)
    return energies


@pytest.mark.parametrize("method", [0, 1, 2, 3, 5])
@pytest.mark.parametrize("n,seed", [(40, 21), (130, 22)])
def test_prefix_methods(ff, oracle_mod, method, n, seed):
    s = synth.make_system(n, seed)
    prefix_or_best(oracle_mod, s, ff, 0, dict(method=method, max_iter=PREFIX))


@pytest.mark.parametrize("ls", [0, 2])
@pytest.mark.parametrize("n,seed", [(40, 21), (130, 22)])
def test_prefix_fgm_restart_option(ff, oracle_mod, n, seed, ls):
    # FGM with the optional function-value momentum restart (Algorithm 1
    # itself, the default, is covered by test_prefix_methods)
    s = synth.make_system(n, seed)
    kw = dict(method=1, ls=ls, max_iter=PREFIX, fgm_restart=1)
    xg, rg, _ = run_gpu(ff, [s], 0, **kw)
    prefix_parity(oracle_mod, s, xg[0], rg[0], kw)


def test_fgm_literal_long_run_returns_best_point(ff, oracle_mod):
    # Algorithm 1 as printed is non-monotone and, from these clashing starts,
    # does not converge (beta -> 1, steps of tens of A); beyond the prefix the
    # GPU and oracle trajectories separate, but the GPU must return its best
    # point with that point's energy, at least as good as the oracle's best
    # point over the first 60 steps (where both take the same steps)
    s = synth.make_system(40, 21)
    kw = dict(method=1, max_iter=400)
    xg, rg, _ = run_gpu(ff, [s], 0, **kw)
    r = rg[0]
    assert r["status_name"] == "max_iter" and r["iterations"] == 400, r
    e1, g1 = oracle_mod.energy_grad(s, xg[0])
    assert abs(e1 - r["energy"]) <= 1e-9 * abs(e1)
    assert abs(np.abs(g1).max() - r["grad_inf"]) <= 1e-9 * np.abs(g1).max()
    xo, ro = oracle_mod.minimize(s, s.x, **dict(kw, max_iter=PREFIX))
    assert r["energy"] <= ro["energy"] * (1 + 1e-8)


@pytest.mark.parametrize("variant", range(7))
def test_prefix_cg_variants(ff, oracle_mod, variant):
    s = synth.make_system(60, 23)
    kw = dict(method=2, cg_variant=variant, max_iter=PREFIX, cg_restart_every=50)
    xg, rg, _ = run_gpu(ff, [s], 0, **kw)
    prefix_parity(oracle_mod, s, xg[0], rg[0], kw)


@pytest.mark.parametrize("ls", [1, 2])
@pytest.mark.parametrize("method", [0, 1, 2, 3, 5])
def test_prefix_line_search_choice(ff, oracle_mod, ls, method):
    s = synth.make_system(50, 24)
    prefix_or_best(oracle_mod, s, ff, 0, dict(method=method, ls=ls, max_iter=PREFIX))


@pytest.mark.parametrize("extra", [dict(ls_par_K=4), dict(ls_par_g0=0), dict(lbfgs_m=1),
                                   dict(lbfgs_m=3), dict(lbfgs_m=16, h0=0.02),
                                   dict(k_plus=3.0, k_minus=0.25)])
def test_prefix_options(ff, oracle_mod, extra):
    s = synth.make_system(45, 25)
    kw = dict(method=3, max_iter=PREFIX, **extra)
    xg, rg, _ = run_gpu(ff, [s], 0, **kw)
    prefix_parity(oracle_mod, s, xg[0], rg[0], kw)


def test_prefix_batched(ff, oracle_mod):
    # systems of a batch advance independently: each matches its own oracle run
    systems = [synth.make_system(n, 300 + k) for k, n in enumerate([60, 33, 140, 7, 90, 2])]
    kw = dict(method=3, max_iter=PREFIX)
    xg, rg, _ = run_gpu(ff, systems, 0, **kw)
    for b, s in enumerate(systems):
        prefix_parity(oracle_mod, s, xg[b], rg[b], kw)


def test_prefix_ogm_batched_and_options(ff, oracle_mod):
    # OGM (Section 4, Eq. 11 with a line search): a batch, each system against
    # its own oracle run; and the G0-free search variant
    systems = [synth.make_system(n, 330 + k) for k, n in enumerate([60, 33, 7])]
    kw = dict(method=5, max_iter=PREFIX)
    xg, rg, _ = run_gpu(ff, systems, 0, **kw)
    for b, s in enumerate(systems):
        prefix_parity(oracle_mod, s, xg[b], rg[b], kw)
    kw = dict(method=5, max_iter=PREFIX, ls_par_g0=0)
    xg, rg, _ = run_gpu(ff, systems[:1], 0, **kw)
    prefix_parity(oracle_mod, systems[0], xg[0], rg[0], kw)


@pytest.mark.parametrize("prec", [0, 1])
def test_ogm_long_capped_run(ff, oracle_mod, prec):
    # beyond the prefix the trajectories separate; the run must lower the
    # energy and report the energy of the point it returns (MIXED: from the
    # FP32 pair terms, as the cap ends the FP32 phase)
    s = synth.make_system(150, 31)
    xg, rg, _ = run_gpu(ff, [s], prec, method=5, max_iter=600)
    r = rg[0]
    assert r["status_name"] in ("ok", "max_iter"), r
    e0 = oracle_mod.energy(s, s.x)
    e1, g1 = oracle_mod.energy_grad(s, xg[0])
    assert e1 < 1e-3 * e0
    if prec == 0:
        assert abs(e1 - r["energy"]) <= 1e-9 * abs(e1), (e1, r)
    else:  # the energy bar of the FP32 pair terms, relative to sum |terms|
        terms = oracle_mod.energy_terms(s, xg[0])[0]
        assert abs(e1 - r["energy"]) <= 1e-5 * terms["sum_abs"], (e1, r)


@pytest.mark.parametrize("beta", [0.0, 0.5, 0.9])
def test_heavy_ball_prefix(ff, oracle_mod, beta):
    # the heavy-ball method of Section 4 (Eq. 8, constant alpha and beta, no
    # line search) from a partly relaxed start, where alpha = 1e-4 is inside
    # the stable range: the same iterates as the oracle's
    s = synth.make_system(80, 45)
    s.x, _ = oracle_mod.minimize(s, s.x, method=3, max_iter=300)
    kw = dict(method=6, hb_alpha=1e-4, hb_beta=beta, max_iter=PREFIX)
    xg, rg, _ = run_gpu(ff, [s], 0, **kw)
    prefix_parity(oracle_mod, s, xg[0], rg[0], kw)


def test_heavy_ball_batched_and_mixed(ff, oracle_mod):
    # a batch of 9 systems (the per-system reduction path) against their own
    # oracle runs; then a MIXED capped run lowers the energy and reports the
    # energy of its returned point
    systems = []
    for k in range(9):
        s = synth.make_system(30 + 11 * k, 340 + k)
        s.x, _ = oracle_mod.minimize(s, s.x, method=3, max_iter=200)
        systems.append(s)
    kw = dict(method=6, hb_alpha=1e-4, hb_beta=0.6, max_iter=PREFIX)
    xg, rg, _ = run_gpu(ff, systems, 0, **kw)
    for b, s in enumerate(systems):
        prefix_parity(oracle_mod, s, xg[b], rg[b], kw)
    s = systems[-1]
    xg, rg, _ = run_gpu(ff, [s], 1, method=6, hb_alpha=1e-4, hb_beta=0.6, max_iter=2000)
    r = rg[0]
    assert r["status_name"] in ("ok", "max_iter"), r
    e0 = oracle_mod.energy(s, s.x)
    e1 = oracle_mod.energy(s, xg[0])
    assert e1 < e0
    terms = oracle_mod.energy_terms(s, xg[0])[0]
    assert abs(e1 - r["energy"]) <= 1e-5 * terms["sum_abs"], (e1, r)


def test_evaluation_cap(ff, oracle_mod):
    s = synth.make_system(30, 29)
    kw = dict(method=3, max_evals=57)
    xg, rg, _ = run_gpu(ff, [s], 0, **kw)
    assert rg[0]["status_name"] == "max_iter"
    prefix_parity(oracle_mod, s, xg[0], rg[0], kw)


@pytest.mark.parametrize("method", [3, 1, 2])
def test_round_limit_timeout(ff, oracle_mod, method):
    # the host-side bound on device rounds (options.max_ticks, a safety net
    # that needs no device-side wait): the run stops with FFMIN_ERR_TIMEOUT
    # after 16 rounds (two graph replays), returning its last accepted point
    # (FGM: its best point) with that point's energy, which is the oracle's
    # point after the same number of accepted steps
    s = synth.make_system(80, 26)
    xg, rg, st = run_gpu(ff, [s], 0, method=method, max_ticks=16)
    r = rg[0]
    assert r["status_name"] == "timeout", r
    assert st["ticks"] == 16
    k = r["iterations"]
    assert k >= 1
    xo, ro = oracle_mod.minimize(s, s.x, method=method, max_iter=k)
    assert np.abs(xg[0] - xo).max() <= 1e-6
    e1, g1 = oracle_mod.energy_grad(s, xg[0])
    assert abs(r["energy"] - e1) <= 1e-9 * abs(e1)
    if np.isfinite(r["grad_inf"]):
        assert abs(r["grad_inf"] - np.abs(g1).max()) <= 1e-9 * np.abs(g1).max()
    else:
        assert method == 1


@pytest.mark.parametrize("prec", [0, 1])
def test_device_loop_equals_host_loop(ff, prec):
    # the single-launch driver (conditional WHILE node) and the host-replayed
    # rounds run the same kernels in the same order: identical results,
    # counts and rounds (batch of 9: the per-system reduction path)
    systems = [synth.make_system(40 + 23 * k, 360 + k) for k in range(9)]
    out = []
    for host_loop in (0, 1):
        S = ff.System(systems, prec)
        x = to_dev([s.x for s in systems])
        r = S.minimize(x, method=3, max_iter=400, host_loop=host_loop)
        out.append((x.cpu().numpy(), r, S.last_stats()["ticks"]))
        S.close()
    (xa, ra, ta), (xb, rb, tb) = out
    assert np.array_equal(xa, xb)
    assert ra == rb
    assert ta == tb


def test_already_converged_start(ff, oracle_mod):
    s = synth.make_system(25, 30)
    xo, ro = oracle_mod.minimize(s, s.x, method=3)
    s.x = xo
    for m in (0, 1, 2, 3, 5):
        xg, rg, _ = run_gpu(ff, [s], 0, method=m)
        assert rg[0]["status_name"] == "ok" and rg[0]["iterations"] == 0 and rg[0]["grad_evals"] == 1


@pytest.mark.parametrize("method", [0, 1, 2, 3])
def test_full_runs_ensemble(ff, oracle_mod, method):
    # FGM with its optional restart: Algorithm 1 as printed does not converge
    # from this start (oracle and GPU alike)
    s = synth.make_system(40, 21)
    kw = dict(method=method, max_iter=100000, fgm_restart=int(method == 1))
    xg, rg, _ = run_gpu(ff, [s], 0, **kw)
    ensemble_parity(oracle_mod, s, xg[0], rg[0], kw)


def test_full_runs_batched_ensemble(ff, oracle_mod):
    systems = [synth.make_system(n, 310 + k) for k, n in enumerate([35, 60, 18])]
    kw = dict(method=3, max_iter=100000)
    xg, rg, _ = run_gpu(ff, systems, 0, **kw)
    for b, s in enumerate(systems):
        ensemble_parity(oracle_mod, s, xg[b], rg[b], kw)


def test_paper_small_config_lbfgs_500(ff, oracle_mod):
    # 500-atom globule (seed 1), L-BFGS m = 10 to |grad|_inf < 0.1: exact for
    # the capped prefix, then compared with a 3-member oracle ensemble
    s = synth.make_system(500, 1)
    kw = dict(method=3, lbfgs_m=10, gtol_inf=0.1, max_iter=PREFIX)
    xg, rg, _ = run_gpu(ff, [s], 0, **kw)
    prefix_parity(oracle_mod, s, xg[0], rg[0], kw)
    kw["max_iter"] = 100000
    xg, rg, _ = run_gpu(ff, [s], 0, **kw)
    ensemble_parity(oracle_mod, s, xg[0], rg[0], kw)


def test_host_entry_point(ff, oracle_mod):
    s = synth.make_system(70, 28)
    S = ff.System([s], 0)
    xh = s.x.reshape(-1).copy()
    r = S.minimize_host(xh, method=3, max_iter=PREFIX)
    S.close()
    prefix_parity(oracle_mod, s, xh.reshape(-1, 3), r[0], dict(method=3, max_iter=PREFIX))


@pytest.mark.parametrize("method", [1, 2, 3])
def test_mixed_fp32_then_fp64(ff, oracle_mod, method):
    # (GD needs more than 1e5 steps on this system in either precision)
    # MIXED: FP32 pair terms until the FP32 run converges or stalls, then the
    # FP64 phase re-evaluates and finishes; the returned point is certified
    # by the oracle's own gradient, and its energy is reported in FP64
    s = synth.make_system(120, 27)
    kw = dict(method=method, max_iter=100000, fgm_restart=int(method == 1))
    xg, rg, _ = run_gpu(ff, [s], 1, **kw)
    r = rg[0]
    assert r["status_name"] == "ok", r
    # a trajectory perturbed at the FP32 scale: held to the fixed ensemble
    # (members perturbed up to 1e-6 A), one-sided at 0.01 %
    ensemble_parity(oracle_mod, s, xg[0], r, kw, mixed=True)


def test_mixed_batched(ff, oracle_mod):
    systems = [synth.make_system(n, 320 + k) for k, n in enumerate([90, 45, 200, 12])]
    kw = dict(method=3, max_iter=100000)
    xg, rg, _ = run_gpu(ff, systems, 1, **kw)
    for b, s in enumerate(systems):
        ensemble_parity(oracle_mod, s, xg[b], rg[b], kw, mixed=True)
