"""Pins of the FP64 oracle's energy and gradient (Section 2 of the paper)
against closed forms, finite differences and invariances, with no GPU."""
import math
import os
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1810_03358_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = int(v, 16) if v.startswith("0x") else float(v)
    return out


def tiny(x, q=None, sigma=None, eps=None, bonds=(), bk=300.0, br0=1.5, angles=(),
         ak=60.0, ath0=None, dih=(), dv=None, c=synth.COULOMB_KCAL):
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    z = np.zeros(n)
    bonds = np.asarray(bonds, dtype=np.int32).reshape(-1, 2)
    angles = np.asarray(angles, dtype=np.int32).reshape(-1, 3)
    dih = np.asarray(dih, dtype=np.int32).reshape(-1, 4)
    return SimpleNamespace(
        x=x, charge=z if q is None else np.asarray(q, float),
        sigma=z + 1.0 if sigma is None else np.asarray(sigma, float),
        epsilon=z if eps is None else np.asarray(eps, float),
        bond_idx=bonds, bond_k=np.full(len(bonds), bk), bond_r0=np.full(len(bonds), br0),
        angle_idx=angles, angle_k=np.full(len(angles), ak),
        angle_theta0=np.zeros(len(angles)) if ath0 is None else np.asarray(ath0, float).reshape(-1),
        dihedral_idx=dih, dihedral_v=np.zeros((len(dih), 4)) if dv is None else np.asarray(dv, float).reshape(-1, 4),
        coulomb_c=c)


def test_coulomb_constant_is_papers(oracle_mod):
    g = golden()
    assert synth.COULOMB_KCAL == pytest.approx(g["coulomb_kj_per_mol"] / g["kj_per_kcal"], rel=1e-15)


def test_two_charges_closed_form(oracle_mod):
    # E_cul = C q1 q2 / r (Section 2); epsilon = 0 removes the LJ term
    for r, q1, q2 in [(3.0, 0.5, -0.7), (7.25, 0.8, 0.8), (1.1, -0.3, 0.45)]:
        s = tiny([[0, 0, 0], [r, 0, 0]], q=[q1, q2])
        d, st, g = oracle_mod.energy_terms(s, s.x, grad=True)
        assert st == 0
        expect = synth.COULOMB_KCAL * q1 * q2 / r
        assert d["coulomb"] == pytest.approx(expect, rel=1e-14)
        assert d["total"] == pytest.approx(expect, rel=1e-14)
        # dE/dx_1 = -C q1 q2 / r^2 along +x for atom 1 (moving it away lowers |E|)
        assert g[1, 0] == pytest.approx(-expect / r, rel=1e-12)
        assert g[0, 0] == pytest.approx(expect / r, rel=1e-12)
        assert d["sum_abs"] == pytest.approx(abs(expect), rel=1e-14)


@pytest.mark.parametrize("si,sj,ei,ej", [(3.0, 3.0, 0.1, 0.1), (2.5, 3.8, 0.02, 0.2)])
def test_lennard_jones_minimum_and_zero(oracle_mod, si, sj, ei, ej):
    # E_vdw = 4 sqrt(ei ej) [(s/r)^12 - (s/r)^6], s = sqrt(si sj): minimum -sqrt(ei ej)
    # at r = 2^(1/6) s, zero at r = s, zero force at the minimum.
    s_ij, e_ij = math.sqrt(si * sj), math.sqrt(ei * ej)
    rmin = 2.0 ** (1.0 / 6.0) * s_ij
    s = tiny([[0, 0, 0], [rmin, 0, 0]], sigma=[si, sj], eps=[ei, ej])
    d, st, g = oracle_mod.energy_terms(s, s.x, grad=True)
    assert d["vdw"] == pytest.approx(-e_ij, rel=1e-13)
    assert np.abs(g).max() < 1e-12
    s = tiny([[0, 0, 0], [s_ij, 0, 0]], sigma=[si, sj], eps=[ei, ej])
    d, st, _ = oracle_mod.energy_terms(s, s.x)
    assert abs(d["vdw"]) < 1e-13
    # one value off the minimum, by hand: r = 1.5 s -> 4e (1.5^-12 - 1.5^-6)
    s = tiny([[0, 0, 0], [1.5 * s_ij, 0, 0]], sigma=[si, sj], eps=[ei, ej])
    d, st, _ = oracle_mod.energy_terms(s, s.x)
    assert d["vdw"] == pytest.approx(4 * e_ij * (1.5 ** -12 - 1.5 ** -6), rel=1e-13)


def test_bond_no_half_factor(oracle_mod):
    # E_stretch = K (r - r0)^2 without a 1/2 (Section 2)
    s = tiny([[0, 0, 0], [1.5, 0, 0]], bonds=[[0, 1]])
    d, _, g = oracle_mod.energy_terms(s, s.x, grad=True)
    assert abs(d["stretch"]) < 1e-20 and np.abs(g).max() < 1e-12
    s = tiny([[0, 0, 0], [1.7, 0, 0]], bonds=[[0, 1]])
    d, _, g = oracle_mod.energy_terms(s, s.x, grad=True)
    assert d["stretch"] == pytest.approx(300.0 * 0.2 ** 2, rel=1e-12)
    assert g[1, 0] == pytest.approx(2 * 300.0 * 0.2, rel=1e-12)


def test_angle_closed_form(oracle_mod):
    # E_bend = K_theta (theta - theta0)^2, no 1/2; vertex is the middle atom
    th = math.radians(109.0)
    x = [[1.2, 0, 0], [0, 0, 0], [1.4 * math.cos(th), 1.4 * math.sin(th), 0]]
    s = tiny(x, angles=[[0, 1, 2]], ath0=[th])
    d, _, g = oracle_mod.energy_terms(s, s.x, grad=True)
    assert abs(d["bend"]) < 1e-20 and np.abs(g).max() < 1e-10
    s = tiny(x, angles=[[0, 1, 2]], ath0=[th - 0.1])
    d, _, _ = oracle_mod.energy_terms(s, s.x)
    assert d["bend"] == pytest.approx(60.0 * 0.1 ** 2, rel=1e-10)


def dihedral_atoms(phi):
    # j-k along z; i and l project onto the xy plane at angle 0 and phi
    return [[1.0, 0.0, -0.5], [0, 0, 0], [0, 0, 1.5], [math.cos(phi), math.sin(phi), 2.0]]


@pytest.mark.parametrize("phi", [0.0, math.pi, math.pi / 2, math.pi / 3, -2.0])
def test_torsion_values(oracle_mod, phi):
    v = [0.7, 0.3, 0.55, 0.2]
    s = tiny(dihedral_atoms(phi), dih=[[0, 1, 2, 3]], dv=[v])
    d, _, _ = oracle_mod.energy_terms(s, s.x)
    c = math.cos
    # closed forms: phi = 0 -> V1 + V3; phi = pi -> 0; general by hand
    if phi == 0.0:
        assert d["torsion"] == pytest.approx(v[0] + v[2], rel=1e-13)
    if phi == math.pi:
        assert abs(d["torsion"]) < 1e-13
    if phi == math.pi / 2:
        assert d["torsion"] == pytest.approx((v[0] + v[2]) / 2 + v[1], rel=1e-13)
    expect = 0.5 * (v[0] * (1 + c(phi)) + v[1] * (1 - c(2 * phi)) + v[2] * (1 + c(3 * phi))
                    + v[3] * (1 - c(4 * phi)))
    assert d["torsion"] == pytest.approx(expect, rel=1e-12, abs=1e-14)


def test_collinear_dihedral_degenerate(oracle_mod):
    x = [[0, 0, -1.5], [0, 0, 0], [0, 0, 1.5], [1.0, 0, 2.5]]
    s = tiny(x, dih=[[0, 1, 2, 3]], dv=[[0.5, 0.2, 0.3, 0.1]])
    d, st, g = oracle_mod.energy_terms(s, s.x, grad=True)
    assert st == 0 and d["degenerate_dihedrals"] == 1
    assert np.abs(g).max() == 0.0
    assert d["torsion"] == pytest.approx(0.5 + 0.3)  # phi = atan2(0, 0) = 0


def test_coincident_atoms_flagged(oracle_mod):
    s = tiny([[1, 2, 3], [1, 2, 3], [4, 0, 0]], q=[0.1, 0.2, 0.3])
    _, st, _ = oracle_mod.energy_terms(s, s.x)
    assert st == 1


def fd_grad(oracle_mod, s, x, h=1e-5):
    x = x.reshape(-1)
    out = np.zeros_like(x)
    for k in range(x.size):
        xp = x.copy(); xp[k] += h
        xm = x.copy(); xm[k] -= h
        out[k] = (oracle_mod.energy(s, xp) - oracle_mod.energy(s, xm)) / (2 * h)
    return out.reshape(-1, 3)


def term_only(s, which):
    t = SimpleNamespace(**vars(s))
    if which != "coulomb":
        t.charge = np.zeros_like(s.charge)
    if which != "vdw":
        t.epsilon = np.zeros_like(s.epsilon)
    if which != "bonds":
        t.bond_idx = s.bond_idx[:0]; t.bond_k = s.bond_k[:0]; t.bond_r0 = s.bond_r0[:0]
    if which != "angles":
        t.angle_idx = s.angle_idx[:0]; t.angle_k = s.angle_k[:0]; t.angle_theta0 = s.angle_theta0[:0]
    if which != "dihedrals":
        t.dihedral_idx = s.dihedral_idx[:0]; t.dihedral_v = s.dihedral_v[:0]
    return t


@pytest.mark.parametrize("which", ["coulomb", "vdw", "bonds", "angles", "dihedrals", "all"])
@pytest.mark.parametrize("n,seed", [(12, 5), (20, 6)])
def test_gradient_central_differences(oracle_mod, which, n, seed):
    s = synth.make_system(n, seed)
    if which != "all":
        s = term_only(s, which)
    e, g = oracle_mod.energy_grad(s, s.x)
    fd = fd_grad(oracle_mod, s, s.x)
    scale = max(np.abs(g).max(), 1e-3)
    assert np.abs(fd - g).max() / scale < 2e-7


@pytest.mark.parametrize("n,seed", [(15, 3), (40, 4)])
def test_translation_rotation_invariance(oracle_mod, n, seed):
    s = synth.make_system(n, seed)
    e0, g = oracle_mod.energy_grad(s, s.x)
    fmax = np.abs(g).max()
    # net force and net torque vanish (E invariant under translation / rotation)
    assert np.abs(g.sum(0)).max() < 1e-10 * max(fmax, 1.0) * n
    torque = np.cross(s.x, g).sum(0)
    assert np.abs(torque).max() < 1e-10 * max(fmax, 1.0) * n * np.abs(s.x).max()
    rng = np.random.default_rng(seed)
    R, t = synth.rigid_motion(rng)
    e1 = oracle_mod.energy(s, s.x @ R.T + t)
    d, _, _ = oracle_mod.energy_terms(s, s.x)
    assert abs(e1 - e0) < 1e-12 * d["sum_abs"]


def test_row_energy_equals_full_difference(oracle_mod):
    s = synth.make_system(9, 11)
    rng = np.random.default_rng(0)
    for i in range(9):
        p = s.x[i] + rng.normal(scale=0.2, size=3)
        x2 = s.x.copy(); x2[i] = p
        full = oracle_mod.energy(s, x2) - oracle_mod.energy(s, s.x)
        row = oracle_mod.row_energy(s, s.x, i, p) - oracle_mod.row_energy(s, s.x, i, s.x[i])
        d, _, _ = oracle_mod.energy_terms(s, s.x)
        assert abs(full - row) < 1e-12 * d["sum_abs"]


def test_neighbour_count_brute_force(oracle_mod):
    s = synth.make_system(60, 2)
    for i in (0, 17, 59):
        d = np.linalg.norm(s.x - s.x[i], axis=1)
        assert oracle_mod.neighbour_count(s, s.x, i, 8.0) == int(((d < 8.0).sum()) - 1)


def test_splitmix64_published_values(oracle_mod):
    g = golden()
    assert oracle_mod.splitmix64(0, 0) == g["splitmix64_seed0_out0"]
    assert oracle_mod.splitmix64(0, 1) == g["splitmix64_seed0_out1"]
    picks = [oracle_mod.pick_atom(99, k, 7) for k in range(2000)]
    assert min(picks) == 0 and max(picks) == 6


def test_atom_gradient_equals_full_gradient_row(oracle_mod):
    s = synth.make_system(25, 13)
    e, g = oracle_mod.energy_grad(s, s.x)
    for i in (0, 1, 12, 23, 24):
        assert np.allclose(oracle_mod.atom_gradient(s, s.x, i), g[i], rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("excl", [0, 1])
def test_energy_delta_definition(oracle_mod, excl):
    # the term-by-term difference equals the difference of the two totals
    # (rounding of the totals: ~u sum|terms|), vanishes at xp = x, splits
    # over row blocks, and its slope at h -> 0 is the directional derivative
    # <grad E, r> of the (separately pinned) gradient
    s = synth.make_system(60, 41)
    s.exclusions, s.scale14 = excl, 0.5
    rng = np.random.default_rng(3)
    r = rng.normal(size=s.x.shape)
    r /= np.linalg.norm(r)
    d0, a0, st = oracle_mod.energy_delta(s, s.x, s.x)
    assert st == 0 and d0 == 0.0 and a0 == 0.0
    tot = oracle_mod.energy_terms(s, s.x)[0]
    for h in (1e-3, 0.05, 0.5):
        xp = s.x + h * r
        d, a, st = oracle_mod.energy_delta(s, s.x, xp)
        assert st == 0 and a >= abs(d)
        ref = oracle_mod.energy(s, xp) - oracle_mod.energy(s, s.x)
        assert abs(d - ref) <= 1e-14 * tot["sum_abs"]
        parts = [oracle_mod.energy_delta(s, s.x, xp, rows=(i0, i0 + 17))[0] for i0 in range(0, 60, 17)]
        assert sum(parts) == pytest.approx(d, rel=1e-12, abs=1e-12 * a)
    e, g = oracle_mod.energy_grad(s, s.x)
    slope = float(np.sum(g * r))
    h = 1e-6
    dp = oracle_mod.energy_delta(s, s.x, s.x + h * r)[0]
    dm = oracle_mod.energy_delta(s, s.x, s.x - h * r)[0]
    assert (dp - dm) / (2 * h) == pytest.approx(slope, rel=1e-5)


@pytest.mark.parametrize("excl", [0, 1])
def test_energy_rows_partition(oracle_mod, excl):
    # row blocks of a partition of [0, N) sum to the whole energy and gradient
    s = synth.make_system(70, 42)
    s.exclusions, s.scale14 = excl, 0.5
    d, st, g = oracle_mod.energy_terms(s, s.x, grad=True)
    tot, gsum = 0.0, np.zeros_like(g)
    parts = {k: 0.0 for k in ("stretch", "bend", "torsion", "coulomb", "vdw", "sum_abs")}
    for i0, i1 in [(0, 9), (9, 33), (33, 34), (34, 70)]:
        dd, st2, gg = oracle_mod.energy_rows(s, s.x, i0, i1)
        assert st2 == 0
        tot += dd["total"]
        gsum += gg
        for k in parts:
            parts[k] += dd[k]
    assert tot == pytest.approx(d["total"], rel=1e-12)
    for k in parts:
        assert parts[k] == pytest.approx(d[k], rel=1e-12, abs=1e-12 * d["sum_abs"]), k
    assert np.abs(gsum - g).max() <= 1e-12 * np.abs(g).max()
