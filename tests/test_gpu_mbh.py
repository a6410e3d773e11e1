"""Monotonic basin hopping on the GPU (every system of a batch hops at once:
perturbation kernel, one batched local minimization, per-system keep) against
the oracle's basin hopping, through the C ABI.

With local searches capped at 25 L-BFGS steps both sides stay in the
prefix regime (the same steps up to rounding), so the hop-by-hop decisions
are the oracle's: the same kept hops, points within 1e-6 A, energies within
1e-8, the same iteration and evaluation totals.  Full local searches end in
chaos-dependent minima; there the run must keep a point no higher than its
own first local minimum (hop 0 is the plain local run from the start) and
certified by the oracle's gradient."""
import numpy as np
import pytest

from paper_1810_03358_gb300 import synth
from tests.gpu_util import need_gpu, split, to_dev

pytestmark = pytest.mark.gpu

CAPPED = dict(method=3, lbfgs_m=10, max_iter=25)


@pytest.fixture(scope="module")
def ff():
    return need_gpu()


def gpu_hop(ffmin, systems, prec, hops, step, seed, **kw):
    S = ffmin.System(systems, prec)
    x = to_dev([s.x for s in systems])
    res, acc = S.basin_hop(x, hops, step, seed, **kw)
    S.close()
    return split(x.cpu().numpy(), systems), res, acc


@pytest.mark.parametrize("n,seed", [(40, 61), (60, 62)])
def test_capped_hops_match_oracle(ff, oracle_mod, n, seed):
    s = synth.make_system(n, seed)
    xg, rg, ag = gpu_hop(ff, [s], 0, 6, 0.3, 1234, **CAPPED)
    xo, ro, ao = oracle_mod.basin_hop(s, s.x, 6, 0.3, 1234, **CAPPED)
    assert ag[0] == ao
    for k in ("iterations", "energy_evals", "grad_evals", "ls_failures"):
        assert rg[0][k] == ro[k], (k, rg[0], ro)
    assert abs(rg[0]["energy"] - ro["energy"]) <= 1e-8 * abs(ro["energy"])
    assert np.abs(xg[0] - xo).max() <= 1e-6


def test_capped_hops_batch(ff, oracle_mod):
    # 9 systems hop together (per-system reductions); system b draws its
    # perturbations from seed + b
    systems = [synth.make_system(30 + 7 * k, 640 + k) for k in range(9)]
    xg, rg, ag = gpu_hop(ff, systems, 0, 4, 0.25, 77, **CAPPED)
    for b, s in enumerate(systems):
        xo, ro, ao = oracle_mod.basin_hop(s, s.x, 4, 0.25, 77 + b, **CAPPED)
        assert ag[b] == ao, b
        assert abs(rg[b]["energy"] - ro["energy"]) <= 1e-8 * abs(ro["energy"]), b
        assert np.abs(xg[b] - xo).max() <= 1e-6, b


@pytest.mark.parametrize("prec", [0, 1])
def test_full_hops_keep_a_valid_lower_minimum(ff, oracle_mod, prec):
    s = synth.make_system(36, 63)
    S = ff.System([s], prec)
    x = to_dev([s.x])
    local = S.minimize(x.clone(), method=3)[0]
    res, acc = S.basin_hop(x, 4, 0.4, 5, method=3)
    S.close()
    r = res[0]
    assert r["status_name"] == "ok", r
    assert r["energy"] <= local["energy"] + 1e-12 * abs(local["energy"])
    e, g = oracle_mod.energy_grad(s, x.cpu().numpy().reshape(-1, 3))
    assert abs(e - r["energy"]) <= 1e-9 * abs(e)
    assert np.abs(g).max() < 0.1 * (1 + 1e-6)
    assert r["iterations"] >= local["iterations"]
