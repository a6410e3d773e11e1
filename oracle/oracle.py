"""ctypes front end of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module.  It accepts any object with the attributes of
a synthetic system (x, charge, sigma, epsilon, bond_idx, ...), so it never
imports the CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

GD, FGM, CG, LBFGS, GRADFREE, OGM, HB = 0, 1, 2, 3, 4, 5, 6
CG_PRP, CG_HS, CG_FR, CG_PRP_PLUS, CG_CD, CG_LS, CG_DY = range(7)
LS_DEFAULT, LS_H, LS_PAR = 0, 1, 2
STATUS = {0: "ok", 1: "nonfinite", 2: "linesearch", 3: "max_iter", 4: "bad_arg"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class _FF(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("charge", _dp), ("sigma", _dp), ("epsilon", _dp),
                ("n_bonds", C.c_int32), ("bond_idx", _ip), ("bond_k", _dp), ("bond_r0", _dp),
                ("n_angles", C.c_int32), ("angle_idx", _ip), ("angle_k", _dp),
                ("angle_theta0", _dp), ("n_dihedrals", C.c_int32), ("dihedral_idx", _ip),
                ("dihedral_v", _dp), ("coulomb_c", C.c_double), ("exclusions", C.c_int32),
                ("scale14", C.c_double)]


class _Terms(C.Structure):
    _fields_ = [("stretch", C.c_double), ("bend", C.c_double), ("torsion", C.c_double),
                ("coulomb", C.c_double), ("vdw", C.c_double), ("total", C.c_double),
                ("sum_abs", C.c_double), ("degenerate_dihedrals", C.c_int32)]


class _Opt(C.Structure):
    _fields_ = [("method", C.c_int32), ("cg_variant", C.c_int32), ("ls", C.c_int32),
                ("lbfgs_m", C.c_int32), ("gtol_inf", C.c_double), ("max_iter", C.c_int32),
                ("max_evals", C.c_int32), ("cg_restart_every", C.c_int32), ("h0", C.c_double),
                ("k_plus", C.c_double), ("k_minus", C.c_double), ("eps_h", C.c_double),
                ("ls_par_K", C.c_int32), ("ls_par_g0", C.c_int32),
                ("gradfree_delta", C.c_double), ("seed", C.c_uint64), ("gradfree_parts", C.c_int32),
                ("gradfree_margin", C.c_double), ("gradfree_taylor_r", C.c_double), ("precond_d", _dp),
                ("mlp_w", _dp), ("ogm_step", C.c_double), ("hb_alpha", C.c_double),
                ("hb_beta", C.c_double), ("fgm_restart", C.c_int32), ("fgm_step", C.c_double),
                ("pc_window", C.c_int32), ("pc_rel", C.c_double), ("pc_gfar", C.c_double)]


class _Res(C.Structure):
    _fields_ = [("energy", C.c_double), ("grad_inf", C.c_double), ("iterations", C.c_int32),
                ("energy_evals", C.c_int32), ("grad_evals", C.c_int32),
                ("ls_failures", C.c_int32), ("status", C.c_int32)]


FG_FN = C.CFUNCTYPE(C.c_double, C.c_void_p, _dp, _dp, _ip)
LINE_FN = C.CFUNCTYPE(C.c_double, C.c_void_p, C.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_energy_terms.argtypes = [C.POINTER(_FF), _dp, _dp, C.POINTER(_Terms)]
        L.orc_energy_terms.restype = C.c_int
        L.orc_energy_rows.argtypes = [C.POINTER(_FF), _dp, C.c_int32, C.c_int32, _dp, C.POINTER(_Terms)]
        L.orc_energy_rows.restype = C.c_int
        L.orc_energy_delta.argtypes = [C.POINTER(_FF), _dp, _dp, C.c_int32, C.c_int32, _dp, _dp]
        L.orc_energy_delta.restype = C.c_int
        L.orc_row_energy.argtypes = [C.POINTER(_FF), _dp, C.c_int32, _dp]
        L.orc_row_energy.restype = C.c_double
        L.orc_row_energy_taylor.argtypes = [C.POINTER(_FF), _dp, C.c_int32, _dp, C.c_double]
        L.orc_row_energy_taylor.restype = C.c_double
        L.orc_atom_gradient.argtypes = [C.POINTER(_FF), _dp, C.c_int32, _dp]
        L.orc_atom_gradient.restype = C.c_int
        L.orc_neighbour_count.argtypes = [C.POINTER(_FF), _dp, C.c_int32, C.c_double]
        L.orc_neighbour_count.restype = C.c_int32
        L.orc_ls_h.argtypes = [LINE_FN, C.c_void_p, C.c_double, C.c_double, C.c_double,
                               C.c_double, C.c_double, _dp, _ip]
        L.orc_ls_h.restype = C.c_double
        L.orc_ls_par.argtypes = [LINE_FN, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                 C.c_int32, C.c_int32, C.c_double, _dp, _ip]
        L.orc_ls_par.restype = C.c_double
        L.orc_options_default.argtypes = [C.POINTER(_Opt)]
        L.orc_minimize.argtypes = [C.c_int32, FG_FN, C.c_void_p, _dp, C.POINTER(_Opt),
                                   C.POINTER(_Res)]
        L.orc_minimize_ff.argtypes = [C.POINTER(_FF), _dp, C.POINTER(_Opt), C.POINTER(_Res)]
        L.orc_basin_hop.argtypes = [C.c_int32, FG_FN, C.c_void_p, _dp, C.POINTER(_Opt), C.c_int32, C.c_double,
                                    C.c_uint64, C.POINTER(_Res), _ip]
        L.orc_basin_hop_ff.argtypes = [C.POINTER(_FF), _dp, C.POINTER(_Opt), C.c_int32, C.c_double, C.c_uint64,
                                       C.POINTER(_Res), _ip]
        L.orc_trace.argtypes = [_dp, _dp, _dp, _dp, C.c_int32]
        L.orc_trace.restype = C.c_int32
        L.orc_lbfgs_direction.argtypes = [C.c_int32, _dp, C.c_int32, _dp, _dp, _dp, _dp]
        L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_pick_atom.argtypes = [C.c_uint64, C.c_uint64, C.c_int32]
        L.orc_pick_atom.restype = C.c_int32
        if hasattr(L, "orc_mlp_forward"):
            _bind_mlp(L)
        _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class FF:
    """Force field of one system, holding its arrays alive for the C side."""

    def __init__(self, s):
        self.keep = dict(
            charge=_f64(s.charge), sigma=_f64(s.sigma), epsilon=_f64(s.epsilon),
            bond_idx=np.ascontiguousarray(s.bond_idx, dtype=np.int32).reshape(-1),
            bond_k=_f64(s.bond_k), bond_r0=_f64(s.bond_r0),
            angle_idx=np.ascontiguousarray(s.angle_idx, dtype=np.int32).reshape(-1),
            angle_k=_f64(s.angle_k), angle_theta0=_f64(s.angle_theta0),
            dihedral_idx=np.ascontiguousarray(s.dihedral_idx, dtype=np.int32).reshape(-1),
            dihedral_v=_f64(s.dihedral_v).reshape(-1))
        k = self.keep
        self.n = int(k["charge"].shape[0])
        self.s = _FF(self.n, _dptr(k["charge"]), _dptr(k["sigma"]), _dptr(k["epsilon"]),
                     int(k["bond_k"].shape[0]), k["bond_idx"].ctypes.data_as(_ip),
                     _dptr(k["bond_k"]), _dptr(k["bond_r0"]), int(k["angle_k"].shape[0]),
                     k["angle_idx"].ctypes.data_as(_ip), _dptr(k["angle_k"]),
                     _dptr(k["angle_theta0"]), int(k["dihedral_v"].shape[0] // 4),
                     k["dihedral_idx"].ctypes.data_as(_ip), _dptr(k["dihedral_v"]),
                     float(s.coulomb_c), int(getattr(s, "exclusions", 0)),
                     float(getattr(s, "scale14", 0.5)))


def _ff(s):
    return s if isinstance(s, FF) else FF(s)


def energy_terms(s, x, grad=False):
    """Returns (terms dict, status, gradient [N,3] or None)."""
    f = _ff(s)
    xx = _f64(x).reshape(-1)
    g = np.zeros_like(xx) if grad else None
    t = _Terms()
    st = lib().orc_energy_terms(C.byref(f.s), _dptr(xx), _dptr(g), C.byref(t))
    d = {k: getattr(t, k) for k, _ in _Terms._fields_}
    return d, st, (g.reshape(-1, 3) if grad else None)


def energy(s, x):
    d, st, _ = energy_terms(s, x)
    return d["total"]


def energy_grad(s, x):
    d, st, g = energy_terms(s, x, grad=True)
    return d["total"], g


def energy_rows(s, x, i0, i1, grad=True):
    """(terms dict, status, gradient [N, 3] or None) of the pairs with
    i0 <= i < j (bonded terms with i0 == 0)."""
    f = _ff(s)
    xx = _f64(x).reshape(-1)
    g = np.zeros_like(xx) if grad else None
    t = _Terms()
    st = lib().orc_energy_rows(C.byref(f.s), _dptr(xx), int(i0), int(i1), _dptr(g), C.byref(t))
    d = {k: getattr(t, k) for k, _ in _Terms._fields_}
    return d, st, (g.reshape(-1, 3) if grad else None)


def energy_delta(s, x, xp, rows=None):
    """(E(xp) - E(x) summed term by term, sum of |term differences|, status);
    rows = (i0, i1) restricts the pairs to rows i0 <= i < i1 (bonded terms
    only with i0 == 0)."""
    f = _ff(s)
    a = _f64(x).reshape(-1)
    b = _f64(xp).reshape(-1)
    i0, i1 = rows if rows is not None else (0, f.n)
    d = C.c_double()
    sa = C.c_double()
    st = lib().orc_energy_delta(C.byref(f.s), _dptr(a), _dptr(b), int(i0), int(i1), C.byref(d), C.byref(sa))
    return d.value, sa.value, st


def row_energy(s, x, i, p):
    f = _ff(s)
    xx = _f64(x).reshape(-1)
    pp = _f64(p).reshape(3)
    return lib().orc_row_energy(C.byref(f.s), _dptr(xx), int(i), _dptr(pp))


def row_energy_taylor(s, x, i, p, r_far):
    """Row energy of atom i at p with the far Coulomb terms linearised."""
    f = _ff(s)
    xx = _f64(x).reshape(-1)
    pp = _f64(p).reshape(3)
    return lib().orc_row_energy_taylor(C.byref(f.s), _dptr(xx), int(i), _dptr(pp), float(r_far))


def atom_gradient(s, x, i):
    """dE/dx_i of one atom (3,), computed from its own terms only."""
    f = _ff(s)
    xx = _f64(x).reshape(-1)
    g = np.zeros(3)
    lib().orc_atom_gradient(C.byref(f.s), _dptr(xx), int(i), _dptr(g))
    return g


def neighbour_count(s, x, i, rc=8.0):
    f = _ff(s)
    xx = _f64(x).reshape(-1)
    return lib().orc_neighbour_count(C.byref(f.s), _dptr(xx), int(i), float(rc))


def options(**kw):
    o = _Opt()
    lib().orc_options_default(C.byref(o))
    keep = None
    keep = []
    for k, v in kw.items():
        if k in ("precond_d", "mlp_w"):
            arr = _f64(v) if v is not None else None
            keep.append(arr)
            setattr(o, k, _dptr(arr))
        else:
            setattr(o, k, v)
    return o, keep


def _result(r):
    d = {k: getattr(r, k) for k, _ in _Res._fields_}
    d["status_name"] = STATUS.get(d["status"], "?")
    return d


def minimize(s, x, **kw):
    """Minimize the force field from x; returns (x_final [N,3], result dict)."""
    f = _ff(s)
    xx = _f64(x).reshape(-1).copy()
    o, keep = options(**kw)
    r = _Res()
    lib().orc_minimize_ff(C.byref(f.s), _dptr(xx), C.byref(o), C.byref(r))
    return xx.reshape(-1, 3), _result(r)


def minimize_fn(fg, x0, **kw):
    """Minimize a Python objective fg(x) -> (f, g) (g may be None when not asked).

    fg(x, want_grad) must return (f, grad or None)."""
    n = int(np.asarray(x0).size)
    xx = _f64(x0).reshape(-1).copy()

    def cb(ctx, xp, gp, st):
        xv = np.ctypeslib.as_array(xp, shape=(n,)).copy()
        want = bool(gp)
        f, g = fg(xv, want)
        if want:
            ga = np.ctypeslib.as_array(gp, shape=(n,))
            ga[:] = g
        st[0] = 0 if np.isfinite(f) else 1
        return float(f)

    cfun = FG_FN(cb)
    o, keep = options(**kw)
    r = _Res()
    lib().orc_minimize(n, cfun, None, _dptr(xx), C.byref(o), C.byref(r))
    return xx, _result(r)


def basin_hop(s, x, hops, step, seed, **kw):
    """Monotonic basin hopping on the force field; returns (x [N,3], result
    dict, accepted hops)."""
    f = _ff(s)
    xx = _f64(x).reshape(-1).copy()
    o, keep = options(**kw)
    r = _Res()
    acc = C.c_int32()
    lib().orc_basin_hop_ff(C.byref(f.s), _dptr(xx), C.byref(o), int(hops), float(step), int(seed), C.byref(r),
                           C.byref(acc))
    return xx.reshape(-1, 3), _result(r), acc.value


def basin_hop_fn(fg, x0, hops, step, seed, **kw):
    """Monotonic basin hopping on a Python objective (as minimize_fn)."""
    n = int(np.asarray(x0).size)
    xx = _f64(x0).reshape(-1).copy()

    def cb(ctx, xp, gp, st):
        xv = np.ctypeslib.as_array(xp, shape=(n,)).copy()
        want = bool(gp)
        f, g = fg(xv, want)
        if want:
            ga = np.ctypeslib.as_array(gp, shape=(n,))
            ga[:] = g
        st[0] = 0 if np.isfinite(f) else 1
        return float(f)

    cfun = FG_FN(cb)
    o, keep = options(**kw)
    r = _Res()
    acc = C.c_int32()
    lib().orc_basin_hop(n, cfun, None, _dptr(xx), C.byref(o), int(hops), float(step), int(seed), C.byref(r),
                        C.byref(acc))
    return xx, _result(r), acc.value


def trace(cap=200000):
    f = np.zeros(cap); h = np.zeros(cap); th = np.zeros(cap); b = np.zeros(cap)
    n = lib().orc_trace(_dptr(f), _dptr(h), _dptr(th), _dptr(b), cap)
    return dict(f=f[:n], h=h[:n], theta=th[:n], beta=b[:n])


def _line(phi):
    calls = []

    def cb(ctx, h):
        calls.append(float(h))
        return float(phi(float(h)))

    return LINE_FN(cb), calls


def ls_h(phi, f_star, h0, eps_h=1e-10, k_plus=2.0, k_minus=0.5):
    """Returns (h, f, list of evaluated h)."""
    cf, calls = _line(phi)
    fo = C.c_double(); ne = C.c_int32()
    h = lib().orc_ls_h(cf, None, f_star, h0, eps_h, k_plus, k_minus, C.byref(fo), C.byref(ne))
    return h, fo.value, calls


def ls_par(phi, f_star, slope, h0, K=2, g0=1, k_plus=2.0):
    cf, calls = _line(phi)
    fo = C.c_double(); ne = C.c_int32()
    h = lib().orc_ls_par(cf, None, f_star, slope, h0, K, g0, k_plus, C.byref(fo), C.byref(ne))
    return h, fo.value, calls


def lbfgs_direction(g, S, Y, d=None):
    """S, Y: [count, n] oldest first."""
    g = _f64(g).reshape(-1)
    n = g.size
    S = _f64(S).reshape(-1, n) if len(S) else np.zeros((0, n))
    Y = _f64(Y).reshape(-1, n) if len(Y) else np.zeros((0, n))
    r = np.zeros(n)
    dd = _f64(d) if d is not None else None
    lib().orc_lbfgs_direction(n, _dptr(g), S.shape[0], _dptr(S), _dptr(Y), _dptr(dd), _dptr(r))
    return r


def splitmix64(seed, k):
    return lib().orc_splitmix64(seed, k)


def pick_atom(seed, k, n):
    return lib().orc_pick_atom(seed, k, n)


def _bind_mlp(L):
    L.orc_mlp_forward.argtypes = [_dp, _dp, _dp]
    L.orc_mlp_forward.restype = C.c_double
    L.orc_mlp_loss_grad.argtypes = [_dp, _dp, _dp, C.c_int64, _dp]
    L.orc_mlp_loss_grad.restype = C.c_double
    L.orc_mlp_features.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int32, C.c_double, _dp]
    L.orc_mlp_features.restype = None


def mlp_forward(w, f):
    w = _f64(w); f = _f64(f)
    return lib().orc_mlp_forward(_dptr(w), _dptr(f), None)


def mlp_loss_grad(w, feat, target):
    w = _f64(w); feat = _f64(feat).reshape(-1, 5); target = _f64(target).reshape(-1)
    g = np.zeros(449)
    loss = lib().orc_mlp_loss_grad(_dptr(w), _dptr(feat), _dptr(target), target.size, _dptr(g))
    return loss, g


def mlp_features(q, sigma, eps, n8, gnorm):
    f = np.zeros(5)
    lib().orc_mlp_features(float(q), float(sigma), float(eps), int(n8), float(gnorm), _dptr(f))
    return f
