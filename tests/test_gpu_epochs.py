"""GPU parity of the parallel-epoch gradient-free search (the parallel form
of Section 3's random-atom moves: parts cut by recursive bisection, one CUDA
block per part on its own copy of the positions) with the FP64 oracle,
through the C ABI.  The host cuts the parts by the same rules as the
oracle; every move takes the same decision as the oracle's (row energies
that differ only in summation order), so the coordinates after K moves
agree to the parabola vertices' rounding."""
import dataclasses

import numpy as np
import pytest

from paper_1810_03358_gb300 import synth
from tests.gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ff():
    return need_gpu()


def run(ffmin, s, prec, **kw):
    S = ffmin.System([s], prec)
    x = to_dev([s.x])
    r = S.minimize(x, **kw)[0]
    st = S.last_stats()
    S.close()
    return x.cpu().numpy().reshape(-1, 3), r, st


@pytest.mark.parametrize("n,P,margin,moves", [(60, 1, 0.0, 150), (130, 2, 0.5, 300), (300, 4, 0.5, 700),
                                              (300, 8, 1.0, 900), (500, 16, 0.5, 1500)])
def test_epochs_match_oracle(ff, oracle_mod, n, P, margin, moves):
    s = synth.make_system(n, 800 + n)
    kw = dict(method=4, max_iter=moves, gtol_inf=1e-9, seed=99, gradfree_delta=0.05,
              gradfree_parts=P, gradfree_margin=margin)
    xg, rg, _ = run(ff, s, 0, **kw)
    xo, ro = oracle_mod.minimize(s, s.x, **kw)
    for k in ("iterations", "energy_evals", "grad_evals"):
        assert rg[k] == ro[k], (k, rg, ro)
    assert rg["status_name"] == ro["status_name"] == "max_iter"
    # same decision at every move (another choice moves an atom by ~delta);
    # a vertex carries the rounding of its row-energy differences divided by
    # the parabola's curvature (measured up to 2e-9 A)
    assert np.abs(xg - xo).max() < 1e-8
    assert abs(rg["energy"] - ro["energy"]) <= 1e-10 * abs(ro["energy"])


def test_one_part_equals_sequential_gpu_path(ff, oracle_mod):
    s = synth.make_system(90, 830)
    kw = dict(method=4, max_iter=400, gtol_inf=1e-9, seed=7, gradfree_delta=0.05)
    xa, ra, _ = run(ff, s, 0, **kw)
    xb, rb, _ = run(ff, s, 0, gradfree_parts=1, **kw)
    assert np.abs(xa - xb).max() < 1e-12
    assert ra["iterations"] == rb["iterations"] and ra["grad_evals"] == rb["grad_evals"]


def test_epochs_with_exclusions(ff, oracle_mod):
    s = dataclasses.replace(synth.make_system(200, 831), exclusions=1, scale14=0.5)
    kw = dict(method=4, max_iter=600, gtol_inf=1e-9, seed=5, gradfree_delta=0.05,
              gradfree_parts=4, gradfree_margin=0.5)
    xg, rg, _ = run(ff, s, 0, **kw)
    xo, ro = oracle_mod.minimize(s, s.x, **kw)
    assert rg["iterations"] == ro["iterations"]
    # vertices carry the rounding of the cancelled excluded clashes (1e-16 of
    # up to 1e10 kcal/mol in every row energy) over small curvatures; a
    # different decision would move an atom by ~delta = 0.05 A
    assert np.abs(xg - xo).max() < 1e-4
    # the reported energy is that of the returned point (within the rounding
    # of the all-pairs sums), and within 1e-6 of the oracle's (the vertices'
    # 1e-5 A times forces of 1e4 kcal/mol/A)
    d0 = oracle_mod.energy_terms(dataclasses.replace(s, exclusions=0), xg)[0]
    assert abs(rg["energy"] - oracle_mod.energy(s, xg)) <= 2e-11 * d0["sum_abs"]
    assert abs(rg["energy"] - ro["energy"]) <= 1e-6 * abs(ro["energy"])


def test_mixed_epochs_lower_the_energy(ff, oracle_mod):
    s = synth.make_system(400, 832)
    e0 = oracle_mod.energy(s, s.x)
    xg, rg, _ = run(ff, s, 1, method=4, max_iter=400 * 10, gtol_inf=0.1, seed=3, gradfree_delta=0.05,
                    gradfree_parts=16, gradfree_margin=0.5)
    e1 = oracle_mod.energy(s, xg)
    assert e1 < 1e-2 * e0
    terms = oracle_mod.energy_terms(s, xg)[0]
    assert abs(rg["energy"] - e1) <= 1e-5 * terms["sum_abs"]


def test_invalid_epoch_options(ff):
    s = synth.make_system(20, 833)
    S = ff.System([s], 0)
    x = to_dev([s.x])
    with pytest.raises(ff.FfminError):
        S.minimize(x, method=4, gradfree_parts=-1)
    with pytest.raises(ff.FfminError):
        S.minimize(x, method=4, gradfree_parts=2, gradfree_margin=-1.0)
    S.close()


def test_epochs_with_taylor_far_field(ff, oracle_mod):
    # parallel epochs with the linearised far-field Coulomb rows (8 parts,
    # r_far = 7 A): the oracle's decisions move for move
    s = synth.make_system(400, 860)
    kw = dict(method=4, max_iter=1000, gtol_inf=1e-9, seed=31, gradfree_delta=0.05, gradfree_parts=8,
              gradfree_margin=0.5, gradfree_taylor_r=7.0)
    xg, rg, _ = run(ff, s, 0, **kw)
    xo, ro = oracle_mod.minimize(s, s.x, **kw)
    for k in ("iterations", "energy_evals", "grad_evals"):
        assert rg[k] == ro[k], (k, rg, ro)
    assert np.abs(xg - xo).max() < 1e-8
