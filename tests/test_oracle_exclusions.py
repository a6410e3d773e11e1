"""Pins of the oracle's exclusion variant (a force-field option outside the
paper, whose Section 2 lets every pair interact): pairs joined by a bond or
by the ends of an angle are excluded, dihedral-end pairs are scaled by
scale14.  Pinned by closed forms, by an independent graph-distance
definition of the excluded pairs, finite differences and invariances."""
import dataclasses
import math
from collections import deque

import numpy as np
import pytest

from paper_1810_03358_gb300 import synth
from tests.test_oracle_energy import fd_grad, tiny


def with_exclusions(s, scale14=0.5):
    if dataclasses.is_dataclass(s):
        return dataclasses.replace(s, exclusions=1, scale14=scale14)
    t = type(s)(**vars(s))
    t.exclusions, t.scale14 = 1, scale14
    return t


def graph_distance(n, bonds):
    adj = [[] for _ in range(n)]
    for i, j in bonds:
        adj[i].append(j)
        adj[j].append(i)
    dist = np.full((n, n), -1, dtype=int)
    for a in range(n):
        dist[a, a] = 0
        q = deque([a])
        while q:
            u = q.popleft()
            for v in adj[u]:
                if dist[a, v] < 0:
                    dist[a, v] = dist[a, u] + 1
                    q.append(v)
    return dist


def pair_energy(oracle_mod, s, i, j):
    """Non-bonded energy of atoms i, j alone (a two-atom system, no terms)."""
    two = tiny(s.x[[i, j]], q=s.charge[[i, j]], sigma=s.sigma[[i, j]], eps=s.epsilon[[i, j]],
               c=s.coulomb_c)
    return oracle_mod.energy(two, two.x)


def test_three_atom_chain_has_no_nonbonded_energy(oracle_mod):
    # bonds (0,1), (1,2) and the angle's ends (0,2) are all excluded: the
    # energy is K (r - r0)^2 per bond plus K_theta (theta - theta0)^2
    x = np.array([[0.0, 0.0, 0.0], [1.6, 0.1, 0.0], [2.1, 1.4, 0.3]])
    s = tiny(x, q=[0.5, -0.3, 0.4], sigma=[3.0, 3.2, 2.9], eps=[0.1, 0.15, 0.05],
             bonds=[(0, 1), (1, 2)], angles=[(0, 1, 2)], ath0=[1.9])
    s = with_exclusions(s)
    u, v = x[0] - x[1], x[2] - x[1]
    theta = math.atan2(np.linalg.norm(np.cross(u, v)), u @ v)
    ref = 300.0 * ((np.linalg.norm(u) - 1.5) ** 2 + (np.linalg.norm(v) - 1.5) ** 2) \
        + 60.0 * (theta - 1.9) ** 2
    assert oracle_mod.energy(s, x) == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("scale14", [0.5, 1.0 / 1.2, 0.0])
@pytest.mark.parametrize("n,seed", [(12, 41), (30, 42)])
def test_excluded_pairs_by_graph_distance(oracle_mod, scale14, n, seed):
    # independent definition: pairs at bond-graph distance 1 or 2 are
    # excluded, distance 3 is scaled (for a chain these are exactly the
    # bond, angle-end and dihedral-end pairs)
    s = synth.make_system(n, seed)
    e_all = oracle_mod.energy(s, s.x)
    dist = graph_distance(n, s.bond_idx)
    corr = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            if dist[i, j] in (1, 2):
                corr -= pair_energy(oracle_mod, s, i, j)
            elif dist[i, j] == 3:
                corr -= (1.0 - scale14) * pair_energy(oracle_mod, s, i, j)
    e_exc = oracle_mod.energy(with_exclusions(s, scale14), s.x)
    d, _, _ = oracle_mod.energy_terms(s, s.x)
    assert abs(e_exc - (e_all + corr)) <= 1e-13 * d["sum_abs"]


@pytest.mark.parametrize("n,seed", [(12, 43), (20, 44)])
def test_gradient_central_differences(oracle_mod, n, seed):
    s = with_exclusions(synth.make_system(n, seed))
    e, g = oracle_mod.energy_grad(s, s.x)
    fd = fd_grad(oracle_mod, s, s.x)
    assert np.abs(fd - g).max() / max(np.abs(g).max(), 1e-3) < 2e-7


def test_invariances_and_row_functions(oracle_mod):
    s = with_exclusions(synth.make_system(25, 45))
    e0, g = oracle_mod.energy_grad(s, s.x)
    fmax = np.abs(g).max()
    assert np.abs(g.sum(0)).max() < 1e-10 * max(fmax, 1.0) * 25
    R, t = synth.rigid_motion(np.random.default_rng(3))
    d, _, _ = oracle_mod.energy_terms(s, s.x)
    assert abs(oracle_mod.energy(s, s.x @ R.T + t) - e0) < 1e-12 * d["sum_abs"]
    # the one-atom functions of the gradient-free method and the samplers
    rng = np.random.default_rng(1)
    for i in (0, 1, 12, 24):
        p = s.x[i] + rng.normal(scale=0.2, size=3)
        x2 = s.x.copy()
        x2[i] = p
        full = oracle_mod.energy(s, x2) - e0
        row = oracle_mod.row_energy(s, s.x, i, p) - oracle_mod.row_energy(s, s.x, i, s.x[i])
        assert abs(full - row) < 1e-12 * d["sum_abs"]
        assert np.allclose(oracle_mod.atom_gradient(s, s.x, i), g[i], rtol=1e-12, atol=1e-9)


def test_minimizers_converge_with_exclusions(oracle_mod):
    s = with_exclusions(synth.make_system(40, 46))
    e0 = oracle_mod.energy(s, s.x)
    xo, r = oracle_mod.minimize(s, s.x, method=3, max_iter=20000)
    assert r["status_name"] == "ok", r
    e1, g1 = oracle_mod.energy_grad(s, xo)
    assert np.abs(g1).max() < 0.1 and e1 < e0
    assert r["energy"] == pytest.approx(e1, rel=1e-12)
