"""The MIXED form's own checks against the FP64 oracle, through the C ABI.

1. Line-search trials.  Three of every four evaluations of a MIXED L-BFGS
   step are energy-only trials f(x + h r), taken as exact FP32 differences
   of every pair term from the search's base point x (plus the bonded
   terms in FP64).  ffmin_energy_delta returns E(x + h r) - E(x) computed
   exactly that way; the oracle's reference is the term-by-term FP64
   difference sum_terms [term(x + h r) - term(x)].  Bar, relative to
   sum |term differences|: 1e-5 (each pair difference carries ~10 FP32
   roundings of its own, u = 6e-8, and chunk sums) plus the first-order
   effect of the FP32 rounding of the base positions (u |x| per
   coordinate), which every difference inherits through the r^-12 power:
   at most 12 * 2 sqrt(3) u |x|max / r_min relative to itself
   (tests.gpu_util.mixed_position_bound; 2e-5 to 1e-4 at the clashing
   starts, whose closest jittered pairs are 0.3 to 1 A apart).  The FP64
   object's difference of two FP64 totals is held to 4e-11 of sum |terms|.
   Wherever the oracle's difference exceeds the bar the MIXED trial must
   take the same decision (sign), which is what a line search consumes.

2. Gradient-free moves: the MIXED search (FP32 row sums) takes the
   oracle's decisions move for move on a small system, its vertices
   within the FP32 rounding of the row sums."""
import numpy as np
import pytest

from paper_1810_03358_gb300 import synth
from tests.gpu_util import mixed_position_bound, need_gpu, oracle_energy_delta, split, to_dev

pytestmark = pytest.mark.gpu

BAR_MIXED = 1e-5
BAR_FP64 = 4e-11


@pytest.fixture(scope="module")
def ff():
    return need_gpu()


def unit_antigradient(oracle_mod, s, x):
    _, g = oracle_mod.energy_grad(s, x)
    r = -g.reshape(-1)
    return r / np.linalg.norm(r)


def check_deltas(ffmin, oracle_mod, systems, xs, rs, hs, blocks=1, tuning=None):
    """GPU differences in both precisions against the oracle; returns the
    worst MIXED error as a fraction of its bar."""
    worst = 0.0
    x = to_dev(xs)
    r = to_dev(rs)
    S64, S32 = ffmin.System(systems, 0), ffmin.System(systems, 1)
    if tuning is not None:
        S32.set_tuning(*tuning)
    bars = [BAR_MIXED + mixed_position_bound(x) for x in xs]
    try:
        for h in hs:
            d64 = S64.energy_delta(x, r, h)
            d32 = S32.energy_delta(x, r, h)
            for b, s in enumerate(systems):
                xp = xs[b] + h * rs[b].reshape(-1, 3)
                if blocks > 1:
                    dref, aref = oracle_energy_delta(s, xs[b], xp, blocks)
                else:
                    dref, aref, st = oracle_mod.energy_delta(s, xs[b], xp)
                    assert st == 0
                tot = oracle_mod.energy_terms(s, xs[b])[0]["sum_abs"]
                assert abs(d64[b] - dref) <= BAR_FP64 * tot, (h, b, d64[b], dref)
                err = abs(d32[b] - dref) / aref
                assert err <= bars[b], (h, b, d32[b], dref, err, bars[b])
                if abs(dref) > bars[b] * aref:
                    assert np.sign(d32[b]) == np.sign(dref), (h, b)
                worst = max(worst, err / bars[b])
    finally:
        S64.close()
        S32.close()
    return worst


def test_difference_trial_3334(ff, oracle_mod):
    # the 10^4-variable globule at its clashing start, along the normalised
    # antigradient (the first search direction), steps 1e-4 .. 1 A
    s = synth.make_system(3334, 2)
    r = unit_antigradient(oracle_mod, s, s.x)
    w = check_deltas(ff, oracle_mod, [s], [s.x], [r], [1e-4, 1e-3, 1e-2, 0.1, 1.0])
    print(f"3334 atoms: MIXED difference trial error {w:.2f} of its bar")


def test_difference_trial_near_minimum(ff, oracle_mod):
    # near a minimum the searches decide on tiny differences: a random unit
    # direction at an L-BFGS minimum of a 150-atom system
    s = synth.make_system(150, 7)
    xo, _ = oracle_mod.minimize(s, s.x, method=oracle_mod.LBFGS)
    r = np.random.default_rng(5).normal(size=xo.size)
    r /= np.linalg.norm(r)
    w = check_deltas(ff, oracle_mod, [s], [xo], [r], [1e-3, 1e-2, 0.1])
    print(f"near minimum: MIXED difference trial error {w:.2f} of its bar")


@pytest.mark.parametrize("ipt", [1, 2])
def test_difference_trial_batch(ff, oracle_mod, ipt):
    # a ragged batch of 16 systems (the per-system reduction path), both
    # FP32 tile shapes
    sizes = [int(n) for n in synth.batch_sizes(256)[:16]]
    systems = [synth.make_system(min(n, 1200), 1000 + b) for b, n in enumerate(sizes)]
    rs = [unit_antigradient(oracle_mod, s, s.x) for s in systems]
    check_deltas(ff, oracle_mod, systems, [s.x for s in systems], rs, [1e-3, 0.1], tuning=(10, ipt))


def test_difference_trial_30000(ff, oracle_mod):
    # the paper-scale globule in the benchmark's configuration, one step of
    # 0.01 A along a random unit direction (oracle rows over the pool)
    s = synth.make_system(30000, 3)
    r = np.random.default_rng(9).normal(size=s.x.size)
    r /= np.linalg.norm(r)
    w = check_deltas(ff, oracle_mod, [s], [s.x], [r], [0.01], blocks=64)
    print(f"30000 atoms: MIXED difference trial error {w:.2f} of its bar")


def test_mixed_gradient_free_decisions(ff, oracle_mod):
    # the MIXED one-atom-at-a-time search on a 40-atom system: same atom
    # sequence (SplitMix64 on both sides) and the same choice at every move;
    # coordinates within the FP32 rounding of the row sums (vertex offsets
    # are row-energy differences over the parabola's curvature)
    s = synth.make_system(40, 44)
    moves = 200
    kw = dict(method=4, max_iter=moves, gtol_inf=1e-12, seed=99, gradfree_delta=0.05)
    S = ff.System([s], 1)
    x = to_dev([s.x])
    rg = S.minimize(x, **kw)
    S.close()
    xg = split(x.cpu().numpy(), [s])[0]
    xo, ro = oracle_mod.minimize(s, s.x, **kw)
    assert rg[0]["iterations"] == ro["iterations"] == moves
    moved_g = np.abs(xg - s.x).max(axis=1) > 0
    moved_o = np.abs(xo - s.x).max(axis=1) > 0
    assert np.array_equal(moved_g, moved_o)
    assert np.abs(xg - xo).max() < 1e-3
