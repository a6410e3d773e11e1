"""Parity of the gradient-free parab moves (Section 3) with the oracle: the
same SplitMix64 atom stream and the same 8-point decision per move, so the
GPU's coordinates after K moves equal the oracle's (the decisions compare
row energies that differ only in summation order)."""
import numpy as np
import pytest

from paper_1810_03358_gb300 import synth
from tests.gpu_util import need_gpu, split, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ff():
    return need_gpu()


@pytest.mark.parametrize("n,moves", [(8, 50), (130, 700), (500, 1200)])
def test_parab_moves_match_oracle(ff, oracle_mod, n, moves):
    s = synth.make_system(n, 400 + n)
    kw = dict(method=4, max_iter=moves, gtol_inf=1e-9, seed=2024, gradfree_delta=0.05)
    S = ff.System([s], 0)
    x = to_dev([s.x])
    r = S.minimize(x, **kw)[0]
    S.close()
    xo, ro = oracle_mod.minimize(s, s.x, **kw)
    assert r["status_name"] == "max_iter" and ro["status_name"] == "max_iter"
    assert r["iterations"] == ro["iterations"] == moves
    assert r["grad_evals"] == ro["grad_evals"]
    xg = x.cpu().numpy().reshape(-1, 3)
    assert np.abs(xg - xo).max() < 1e-9
    assert abs(r["energy"] - ro["energy"]) <= 1e-10 * abs(ro["energy"])


def test_parab_energy_decreases_mixed(ff, oracle_mod):
    s = synth.make_system(300, 410)
    S = ff.System([s], 1)
    x = to_dev([s.x])
    e0 = oracle_mod.energy(s, s.x)
    r = S.minimize(x, method=4, max_iter=900, gtol_inf=1e-9, seed=7)[0]
    S.close()
    e1 = oracle_mod.energy(s, x.cpu().numpy())
    assert r["iterations"] == 900 and e1 < e0
    assert abs(r["energy"] - e1) <= 1e-6 * abs(e1) + 1e-3


@pytest.mark.parametrize("n,moves,r_far", [(130, 700, 6.0), (500, 1200, 8.0), (500, 600, 1e9)])
def test_taylor_far_field_moves_match_oracle(ff, oracle_mod, n, moves, r_far):
    # Section 3's linearised far-field Coulomb rows (atoms at least r_far
    # from the moving atom's current position): the same decisions as the
    # oracle's orc_row_energy_taylor moves; r_far beyond the system is the
    # exact method
    s = synth.make_system(n, 420 + n)
    kw = dict(method=4, max_iter=moves, gtol_inf=1e-9, seed=2025, gradfree_delta=0.05,
              gradfree_taylor_r=r_far)
    S = ff.System([s], 0)
    x = to_dev([s.x])
    r = S.minimize(x, **kw)[0]
    S.close()
    xo, ro = oracle_mod.minimize(s, s.x, **kw)
    assert r["iterations"] == ro["iterations"] == moves
    xg = x.cpu().numpy().reshape(-1, 3)
    assert np.abs(xg - xo).max() < 1e-8
    assert abs(r["energy"] - ro["energy"]) <= 1e-10 * abs(ro["energy"])
    if r_far > 100:
        xe, re_ = oracle_mod.minimize(s, s.x, **dict(kw, gradfree_taylor_r=0.0))
        assert np.abs(xg - xe).max() < 1e-8
