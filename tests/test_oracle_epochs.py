"""Pins of the oracle's parallel-epoch gradient-free search (the parallel
form of the random-atom moves that Section 3 proposes): with one part it is
the sequential method, move for move; with several parts it equals a brute
force that takes every trial energy as a full-energy difference."""
import numpy as np
import pytest

from paper_1810_03358_gb300 import synth


@pytest.mark.parametrize("n,moves", [(9, 9), (9, 31), (40, 80), (40, 97)])
def test_one_part_is_the_sequential_method(oracle_mod, n, moves):
    s = synth.make_system(n, 700 + n)
    kw = dict(method=oracle_mod.GRADFREE, max_iter=moves, gtol_inf=1e-9, seed=5, gradfree_delta=0.05)
    xa, ra = oracle_mod.minimize(s, s.x, **kw)
    xb, rb = oracle_mod.minimize(s, s.x, gradfree_parts=1, gradfree_margin=3.0, **kw)
    assert np.array_equal(xa, xb)
    for k in ("iterations", "energy_evals", "grad_evals", "status"):
        assert ra[k] == rb[k], k
    assert ra["energy"] == rb["energy"]


def partition(oracle_mod, x, e, P, seed):
    """Recursive bisection of the epoch rules: (part of each atom, boxes)."""
    n = x.shape[0]
    part = np.zeros(n, dtype=int)
    boxes = []

    def rec(A, p, lo, hi, node):
        if p == 1:
            for a in A:
                part[a] = len(boxes)
            boxes.append((lo.copy(), hi.copy()))
            return
        ext = x[A].max(0) - x[A].min(0)
        axis = int(np.argmax(ext))  # first of equal extents
        A = sorted(A, key=lambda a: (x[a, axis], a))
        na, p1 = len(A), p // 2
        span = max(1, na // (2 * p))
        c = (2 * na * p1 + p) // (2 * p) + oracle_mod.pick_atom(seed, (1 << 62) + (e << 20) + node, span) - span // 2
        c = min(max(c, 1), na - 1)
        plane = 0.5 * (x[A[c - 1], axis] + x[A[c], axis])
        hl, lr = hi.copy(), lo.copy()
        hl[axis] = plane
        lr[axis] = plane
        rec(A[:c], p1, lo, hl, 2 * node + 1)
        rec(A[c:], p - p1, lr, hi, 2 * node + 2)

    rec(list(range(n)), min(P, n), np.full(3, -np.inf), np.full(3, np.inf), 0)
    return part, boxes


def brute_force_epochs(oracle_mod, s, x, epochs, P, margin, seed, delta):
    """The epoch rules restated with full-energy differences for every trial
    (the oracle uses the one-atom row energy)."""
    x = x.copy()
    n = x.shape[0]
    moves = 0
    for e in range(epochs):
        part, boxes = partition(oracle_mod, x, e, P, seed)
        xs = x.copy()
        for q, (lo, hi) in enumerate(boxes):
            members = [a for a in range(n) if part[a] == q]
            movable = [a for a in members if np.all(xs[a] - lo >= margin) and np.all(hi - xs[a] >= margin)]
            xv = xs.copy()
            for m in range(len(movable)):
                i = movable[oracle_mod.pick_atom(seed, (q << 40) + e * n + m, len(movable))]
                base = oracle_mod.energy(s, xv)
                pts = [xv[i].copy()]
                for a in range(3):
                    for sgn in (1, -1):
                        p = xv[i].copy()
                        p[a] += sgn * delta
                        pts.append(p)

                def de(p):
                    y = xv.copy()
                    y[i] = p
                    return oracle_mod.energy(s, y) - base

                f = [de(p) for p in pts]
                v = xv[i].copy()
                for a in range(3):
                    fp, fm = f[1 + 2 * a], f[2 + 2 * a]
                    curv = fm - 2 * f[0] + fp
                    v[a] += delta * (fm - fp) / (2 * curv) if curv > 0 else 0.0
                pts.append(v)
                f.append(de(v))
                xv[i] = pts[int(np.argmin(f))]
            for a in members:
                x[a] = xv[a]
            moves += len(movable)
    return x, moves


@pytest.mark.parametrize("P,margin,n", [(2, 0.5, 14), (3, 0.3, 16), (4, 0.2, 20)])
def test_parts_match_brute_force(oracle_mod, P, margin, n):
    s = synth.make_system(n, 710 + P)
    x_bf, total = brute_force_epochs(oracle_mod, s, s.x, 2, P, margin, 11, 0.05)
    assert total > 0
    xo, ro = oracle_mod.minimize(s, s.x, method=oracle_mod.GRADFREE, max_iter=total, gtol_inf=1e-9,
                                 seed=11, gradfree_delta=0.05, gradfree_parts=P, gradfree_margin=margin)
    assert ro["iterations"] == total
    assert np.abs(xo - x_bf).max() < 1e-9


def test_epochs_lower_the_energy(oracle_mod):
    s = synth.make_system(80, 720)
    e0 = oracle_mod.energy(s, s.x)
    xo, ro = oracle_mod.minimize(s, s.x, method=oracle_mod.GRADFREE, max_iter=80 * 20, gtol_inf=0.1,
                                 seed=3, gradfree_delta=0.05, gradfree_parts=4, gradfree_margin=0.5)
    e1 = oracle_mod.energy(s, xo)
    assert e1 < 1e-2 * e0
    assert ro["energy"] == pytest.approx(e1, rel=1e-12)


@pytest.mark.parametrize("n,P,seed", [(14, 2, 11), (300, 8, 99), (1000, 64, 5), (3334, 128, 3)])
def test_library_host_cut_matches_the_rules(oracle_mod, n, P, seed):
    # the CUDA library cuts the parts on the host: its cut (no GPU needed)
    # equals the rules restated above, which the oracle's moves also match
    from paper_1810_03358_gb300 import build, ffmin
    build.build()
    s = synth.make_system(n, 740 + n)
    for e in (0, 3):
        part, mov = ffmin.ffmin_epoch_parts(s.x, P, seed, e, 0.5)
        ref, boxes = partition(oracle_mod, s.x, e, P, seed)
        assert np.array_equal(part, ref)
        ref_mov = [bool(np.all(s.x[a] - boxes[ref[a]][0] >= 0.5) and np.all(boxes[ref[a]][1] - s.x[a] >= 0.5))
                   for a in range(n)]
        assert np.array_equal(mov, ref_mov)
