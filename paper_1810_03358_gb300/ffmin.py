"""Thin ctypes binding of libffmin.so (the C ABI of include/ffmin.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (FP64, contiguous, [3N] or
[N, 3]); the stream is torch's current stream unless one is given.  There is
no CPU fallback: loading fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libffmin.so")

FFMIN_OK, FFMIN_ERR_INVALID_ARG, FFMIN_ERR_CUDA, FFMIN_ERR_NONFINITE = 0, 1, 2, 3
FFMIN_ERR_LINESEARCH, FFMIN_ERR_MAX_ITER, FFMIN_ERR_TIMEOUT, FFMIN_ERR_OOM = 4, 5, 6, 7
STATUS_NAMES = {0: "ok", 1: "invalid_arg", 2: "cuda", 3: "nonfinite", 4: "linesearch",
                5: "max_iter", 6: "timeout", 7: "oom"}
FFMIN_GD, FFMIN_FGM, FFMIN_CG, FFMIN_LBFGS, FFMIN_GRADFREE, FFMIN_OGM, FFMIN_HB = range(7)
(FFMIN_CG_PRP, FFMIN_CG_HS, FFMIN_CG_FR, FFMIN_CG_PRP_PLUS, FFMIN_CG_CD, FFMIN_CG_LS,
 FFMIN_CG_DY) = range(7)
FFMIN_LS_DEFAULT, FFMIN_LS_H, FFMIN_LS_PAR = range(3)
FFMIN_FP64, FFMIN_MIXED = 0, 1
METHODS = {"GD": FFMIN_GD, "FGM": FFMIN_FGM, "CG": FFMIN_CG, "LBFGS": FFMIN_LBFGS,
           "GRADFREE": FFMIN_GRADFREE, "OGM": FFMIN_OGM, "HB": FFMIN_HB}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class ffmin_topology(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("charge", _dp), ("sigma", _dp), ("epsilon", _dp),
                ("n_bonds", C.c_int32), ("bond_idx", _ip), ("bond_k", _dp), ("bond_r0", _dp),
                ("n_angles", C.c_int32), ("angle_idx", _ip), ("angle_k", _dp),
                ("angle_theta0", _dp), ("n_dihedrals", C.c_int32), ("dihedral_idx", _ip),
                ("dihedral_v", _dp), ("coulomb_c", C.c_double), ("exclusions", C.c_int32),
                ("scale14", C.c_double)]


class ffmin_options(C.Structure):
    _fields_ = [("method", C.c_int32), ("cg_variant", C.c_int32), ("ls", C.c_int32),
                ("lbfgs_m", C.c_int32), ("gtol_inf", C.c_double), ("max_iter", C.c_int32),
                ("max_evals", C.c_int32), ("cg_restart_every", C.c_int32), ("h0", C.c_double),
                ("k_plus", C.c_double), ("k_minus", C.c_double), ("eps_h", C.c_double),
                ("ls_par_K", C.c_int32), ("ls_par_g0", C.c_int32),
                ("gradfree_delta", C.c_double), ("seed", C.c_uint64), ("gradfree_parts", C.c_int32),
                ("gradfree_margin", C.c_double),
                ("use_learned_precond", C.c_int32), ("max_ticks", C.c_int32),
                ("record_dev", C.c_void_p), ("record_every", C.c_int32), ("record_slots", C.c_int32),
                ("fgm_restart", C.c_int32), ("hb_alpha", C.c_double), ("hb_beta", C.c_double),
                ("gradfree_taylor_r", C.c_double), ("host_loop", C.c_int32),
                ("pc_window", C.c_int32), ("pc_rel", C.c_double), ("pc_gfar", C.c_double)]


class ffmin_result(C.Structure):
    _fields_ = [("energy", C.c_double), ("grad_inf", C.c_double), ("iterations", C.c_int32),
                ("energy_evals", C.c_int32), ("grad_evals", C.c_int32),
                ("ls_failures", C.c_int32), ("stop_reason", C.c_int32),
                ("fp64_iterations", C.c_int32)]


EXPORTS = ["ffmin_options_default", "ffmin_status_string", "ffmin_create", "ffmin_destroy",
           "ffmin_n_atoms", "ffmin_atom_offset", "ffmin_energy", "ffmin_energy_grad",
           "ffmin_energy_grad_host", "ffmin_energy_delta", "ffmin_minimize", "ffmin_minimize_host",
           "ffmin_basin_hop",
           "ffmin_set_precond", "ffmin_time_pair_kernel", "ffmin_last_stats",
           "ffmin_last_error", "ffmin_pair_energy_grad_noalloc", "ffmin_neighbour_counts",
           "ffmin_mlp_train", "ffmin_mlp_work_floats", "ffmin_autotune", "ffmin_set_tuning",
           "ffmin_get_tuning", "ffmin_alu_peak",
           "ffmin_epoch_parts"]

_lib = None


def lib():
    """Load libffmin.so; raise if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_1810_03358_gb300.build.build() "
                           "(the CUDA library is required; there is no CPU path)")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.ffmin_options_default.argtypes = [C.POINTER(ffmin_options)]
    L.ffmin_options_default.restype = None
    L.ffmin_status_string.argtypes = [C.c_int]
    L.ffmin_status_string.restype = C.c_char_p
    L.ffmin_create.argtypes = [C.POINTER(ffmin_topology), C.c_int32, C.c_int32, vp, C.POINTER(vp)]
    L.ffmin_destroy.argtypes = [vp]
    L.ffmin_n_atoms.argtypes = [vp]
    L.ffmin_n_atoms.restype = C.c_int64
    L.ffmin_atom_offset.argtypes = [vp, C.c_int32]
    L.ffmin_atom_offset.restype = C.c_int64
    L.ffmin_alu_peak.argtypes = [C.c_int32, C.c_int32, _dp]
    L.ffmin_epoch_parts.argtypes = [_dp, C.c_int32, C.c_int32, C.c_uint64, C.c_uint64, C.c_double, _ip, _ip]
    L.ffmin_energy.argtypes = [vp, vp, _dp]
    L.ffmin_energy_grad.argtypes = [vp, vp, _dp, vp]
    L.ffmin_energy_grad_host.argtypes = [vp, _dp, _dp, _dp]
    L.ffmin_energy_delta.argtypes = [vp, vp, vp, C.c_double, _dp]
    L.ffmin_minimize.argtypes = [vp, vp, C.POINTER(ffmin_options), C.POINTER(ffmin_result)]
    L.ffmin_minimize_host.argtypes = [vp, _dp, C.POINTER(ffmin_options), C.POINTER(ffmin_result)]
    L.ffmin_basin_hop.argtypes = [vp, vp, C.POINTER(ffmin_options), C.c_int32, C.c_double, C.c_uint64,
                                  C.POINTER(ffmin_result), _ip]
    L.ffmin_set_precond.argtypes = [vp, C.POINTER(C.c_uint16), C.c_int32]
    L.ffmin_time_pair_kernel.argtypes = [vp, vp, C.c_int32, C.c_int32, C.POINTER(C.c_float)]
    L.ffmin_last_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.ffmin_pair_energy_grad_noalloc.argtypes = [vp, vp, vp, vp, C.c_int32, C.c_double, vp, vp, vp]
    L.ffmin_neighbour_counts.argtypes = [vp, vp, vp]
    L.ffmin_autotune.argtypes = [vp, vp, C.POINTER(C.c_int32)]
    L.ffmin_set_tuning.argtypes = [vp, C.c_int32, C.c_int32]
    L.ffmin_get_tuning.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.ffmin_mlp_train.argtypes = [vp, vp, C.c_int64, C.c_int32, C.c_int32, C.c_float, C.c_uint64, vp, vp,
                                  vp, C.POINTER(C.c_float), vp, vp]
    L.ffmin_mlp_work_floats.argtypes = []
    L.ffmin_mlp_work_floats.restype = C.c_int64
    L.ffmin_last_error.argtypes = [vp]
    L.ffmin_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("ffmin_options_default", "ffmin_status_string", "ffmin_n_atoms",
                        "ffmin_atom_offset", "ffmin_last_error", "ffmin_mlp_work_floats"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


class FfminError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st, handle=None):
    if st != FFMIN_OK:
        msg = lib().ffmin_last_error(handle)
        raise FfminError(st, msg.decode() if msg else "")


def ffmin_options_default(**overrides) -> ffmin_options:
    o = ffmin_options()
    lib().ffmin_options_default(C.byref(o))
    for k, v in overrides.items():
        if k == "method" and isinstance(v, str):
            v = METHODS[v]
        setattr(o, k, v)
    return o


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _topology(s, keep):
    arrs = dict(
        charge=_f64(s.charge), sigma=_f64(s.sigma), epsilon=_f64(s.epsilon),
        bond_idx=np.ascontiguousarray(s.bond_idx, dtype=np.int32).reshape(-1),
        bond_k=_f64(s.bond_k), bond_r0=_f64(s.bond_r0),
        angle_idx=np.ascontiguousarray(s.angle_idx, dtype=np.int32).reshape(-1),
        angle_k=_f64(s.angle_k), angle_theta0=_f64(s.angle_theta0),
        dihedral_idx=np.ascontiguousarray(s.dihedral_idx, dtype=np.int32).reshape(-1),
        dihedral_v=_f64(s.dihedral_v).reshape(-1))
    keep.append(arrs)
    d = lambda k: arrs[k].ctypes.data_as(_dp)
    i = lambda k: arrs[k].ctypes.data_as(_ip)
    return ffmin_topology(int(arrs["charge"].size), d("charge"), d("sigma"), d("epsilon"),
                          int(arrs["bond_k"].size), i("bond_idx"), d("bond_k"), d("bond_r0"),
                          int(arrs["angle_k"].size), i("angle_idx"), d("angle_k"),
                          d("angle_theta0"), int(arrs["dihedral_v"].size // 4),
                          i("dihedral_idx"), d("dihedral_v"), float(getattr(s, "coulomb_c", 0.0)),
                          int(getattr(s, "exclusions", 0)), float(getattr(s, "scale14", 0.5)))


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def ffmin_create(systems, precision=FFMIN_FP64, stream=None):
    """Create a batch from synthetic systems (objects with the topology
    attributes); returns an opaque handle (int)."""
    if not isinstance(systems, (list, tuple)):
        systems = [systems]
    keep = []
    tops = (ffmin_topology * len(systems))(*[_topology(s, keep) for s in systems])
    h = C.c_void_p()
    st = lib().ffmin_create(tops, len(systems), int(precision), C.c_void_p(_stream_handle(stream)),
                            C.byref(h))
    _check(st, None)
    return h.value


def ffmin_destroy(handle):
    _check(lib().ffmin_destroy(C.c_void_p(handle)))


def ffmin_n_atoms(handle):
    return int(lib().ffmin_n_atoms(C.c_void_p(handle)))


def ffmin_atom_offset(handle, b):
    return int(lib().ffmin_atom_offset(C.c_void_p(handle), int(b)))


def _dev_ptr(t, n_atoms):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if t.numel() != 3 * n_atoms:
        raise ValueError(f"expected {3 * n_atoms} coordinates, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def ffmin_energy(handle, x, n_sys=1):
    e = np.zeros(n_sys)
    st = lib().ffmin_energy(C.c_void_p(handle), _dev_ptr(x, ffmin_n_atoms(handle)),
                            e.ctypes.data_as(_dp))
    _check(st, handle)
    return e


def ffmin_energy_grad(handle, x, g, n_sys=1):
    e = np.zeros(n_sys)
    n = ffmin_n_atoms(handle)
    st = lib().ffmin_energy_grad(C.c_void_p(handle), _dev_ptr(x, n), e.ctypes.data_as(_dp),
                                 _dev_ptr(g, n))
    _check(st, handle)
    return e


def ffmin_energy_grad_host(handle, x_host, g_host=None, n_sys=1):
    e = np.zeros(n_sys)
    x = _f64(x_host).reshape(-1)
    gp = None
    if g_host is not None:
        assert g_host.dtype == np.float64 and g_host.flags.c_contiguous
        gp = g_host.ctypes.data_as(_dp)
    st = lib().ffmin_energy_grad_host(C.c_void_p(handle), x.ctypes.data_as(_dp),
                                      e.ctypes.data_as(_dp), gp)
    _check(st, handle)
    return e


def ffmin_energy_delta(handle, x, r, h, n_sys=1):
    """E(x + h r) - E(x) per system, as a line-search trial evaluates it."""
    de = np.zeros(n_sys)
    n = ffmin_n_atoms(handle)
    st = lib().ffmin_energy_delta(C.c_void_p(handle), _dev_ptr(x, n), _dev_ptr(r, n), float(h),
                                  de.ctypes.data_as(_dp))
    _check(st, handle)
    return de


def _results(rs):
    out = []
    for r in rs:
        d = {k: getattr(r, k) for k, _ in ffmin_result._fields_}
        d["status_name"] = STATUS_NAMES.get(d["stop_reason"], "?")
        out.append(d)
    return out


def ffmin_minimize(handle, x, options, n_sys=1):
    """Minimize in place (x: FP64 CUDA tensor); returns a list of result dicts."""
    rs = (ffmin_result * n_sys)()
    st = lib().ffmin_minimize(C.c_void_p(handle), _dev_ptr(x, ffmin_n_atoms(handle)),
                              C.byref(options), rs)
    _check(st, handle)
    return _results(rs)


def ffmin_basin_hop(handle, x, options, hops, step, seed, n_sys=1):
    """Monotonic basin hopping in place (x: FP64 CUDA tensor); returns
    (list of result dicts, list of accepted hops per system)."""
    rs = (ffmin_result * n_sys)()
    acc = np.zeros(n_sys, dtype=np.int32)
    st = lib().ffmin_basin_hop(C.c_void_p(handle), _dev_ptr(x, ffmin_n_atoms(handle)), C.byref(options),
                               int(hops), float(step), int(seed), rs, acc.ctypes.data_as(_ip))
    _check(st, handle)
    return _results(rs), [int(a) for a in acc]


def ffmin_minimize_host(handle, x_host, options, n_sys=1):
    """x_host: float64 numpy array [3N], minimized in place."""
    assert x_host.dtype == np.float64 and x_host.flags.c_contiguous
    rs = (ffmin_result * n_sys)()
    st = lib().ffmin_minimize_host(C.c_void_p(handle), x_host.ctypes.data_as(_dp),
                                   C.byref(options), rs)
    _check(st, handle)
    return _results(rs)


def ffmin_set_precond(handle, w_fp16):
    w = np.ascontiguousarray(w_fp16, dtype=np.float16).view(np.uint16)
    st = lib().ffmin_set_precond(C.c_void_p(handle), w.ctypes.data_as(C.POINTER(C.c_uint16)),
                                 int(w.size))
    _check(st, handle)


def ffmin_time_pair_kernel(handle, x, with_grad=True, reps=10):
    ms = C.c_float()
    st = lib().ffmin_time_pair_kernel(C.c_void_p(handle), _dev_ptr(x, ffmin_n_atoms(handle)),
                                      int(with_grad), int(reps), C.byref(ms))
    _check(st, handle)
    return ms.value


def ffmin_epoch_parts(x, parts, seed, epoch, margin):
    """Host-side parts of one epoch of the parallel gradient-free search:
    (part of each atom, movable flags) for positions x [N, 3] (numpy)."""
    xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    n = xx.size // 3
    part = np.zeros(n, dtype=np.int32)
    mov = np.zeros(n, dtype=np.int32)
    _check(lib().ffmin_epoch_parts(xx.ctypes.data_as(_dp), n, int(parts), int(seed), int(epoch),
                                   float(margin), part.ctypes.data_as(_ip), mov.ctypes.data_as(_ip)))
    return part, mov.astype(bool)


def ffmin_alu_peak(precision, reps=10):
    """Measured FP32 (precision = FFMIN_MIXED) or FP64 FMA peak, TFLOP/s."""
    t = C.c_double()
    _check(lib().ffmin_alu_peak(int(precision), int(reps), C.byref(t)))
    return t.value


def ffmin_last_stats(handle):
    t, l, p = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().ffmin_last_stats(C.c_void_p(handle), C.byref(t), C.byref(l), C.byref(p)), handle)
    return dict(ticks=t.value, launches=l.value, pair_interactions=p.value)


class System:
    """Owning wrapper: a batch of systems on the GPU."""

    def __init__(self, systems, precision=FFMIN_FP64, stream=None):
        if not isinstance(systems, (list, tuple)):
            systems = [systems]
        self.n_sys = len(systems)
        self.handle = ffmin_create(systems, precision, stream)
        self.n_atoms = ffmin_n_atoms(self.handle)
        self.offsets = [ffmin_atom_offset(self.handle, b) for b in range(self.n_sys + 1)]

    def close(self):
        if self.handle:
            ffmin_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def energy(self, x):
        return ffmin_energy(self.handle, x, self.n_sys)

    def energy_grad(self, x, g=None):
        import torch
        if g is None:
            g = torch.empty_like(x)
        e = ffmin_energy_grad(self.handle, x, g, self.n_sys)
        return e, g

    def energy_delta(self, x, r, h):
        return ffmin_energy_delta(self.handle, x, r, h, self.n_sys)

    def minimize(self, x, **opts):
        o = ffmin_options_default(**opts)
        return ffmin_minimize(self.handle, x, o, self.n_sys)

    def basin_hop(self, x, hops, step, seed, **opts):
        o = ffmin_options_default(**opts)
        return ffmin_basin_hop(self.handle, x, o, hops, step, seed, self.n_sys)

    def minimize_host(self, x_host, **opts):
        o = ffmin_options_default(**opts)
        return ffmin_minimize_host(self.handle, x_host, o, self.n_sys)

    def time_pair_kernel(self, x, with_grad=True, reps=10):
        return ffmin_time_pair_kernel(self.handle, x, with_grad, reps)

    def last_stats(self):
        return ffmin_last_stats(self.handle)

    def autotune(self, x):
        return ffmin_autotune(self.handle, x)

    def set_tuning(self, density, f32_atoms_per_thread):
        ffmin_set_tuning(self.handle, density, f32_atoms_per_thread)

    def get_tuning(self):
        return ffmin_get_tuning(self.handle)


def ffmin_status_string(status):
    return lib().ffmin_status_string(int(status)).decode()


def ffmin_last_error(handle=None):
    m = lib().ffmin_last_error(C.c_void_p(handle) if handle else None)
    return m.decode() if m else ""


def ffmin_pair_energy_grad_noalloc(x, charge, sigma, epsilon, g, e, coulomb_c=0.0, stream=None):
    """Non-bonded E + grad of one system with caller-owned device buffers and
    no allocation inside the library (torch FP64 CUDA tensors: x [3N],
    charge / sigma / epsilon [N], g [3N] out, e [1] out).  Returns the status;
    raises FfminError on failure."""
    import torch
    n = int(charge.numel())

    def per_atom(t, what, count):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise FfminError(FFMIN_ERR_INVALID_ARG, f"{what}: expected a contiguous float64 CUDA tensor")
        if t.numel() != count:
            raise FfminError(FFMIN_ERR_INVALID_ARG, f"{what}: expected {count} values, got {t.numel()}")
        return C.c_void_p(t.data_ptr())

    px, pg = per_atom(x, "x", 3 * n), per_atom(g, "g", 3 * n)
    pq, ps, pe = per_atom(charge, "charge", n), per_atom(sigma, "sigma", n), per_atom(epsilon, "epsilon", n)
    if not (isinstance(e, torch.Tensor) and e.is_cuda and e.dtype == torch.float64 and e.numel() >= 1):
        raise FfminError(FFMIN_ERR_INVALID_ARG, "e: expected a float64 CUDA tensor with at least one value")
    st = lib().ffmin_pair_energy_grad_noalloc(px, pq, ps, pe, n, float(coulomb_c), pg,
                                              C.c_void_p(e.data_ptr()), C.c_void_p(_stream_handle(stream)))
    if st != FFMIN_OK:
        raise FfminError(st, "ffmin_pair_energy_grad_noalloc failed")
    return st


def ffmin_neighbour_counts(handle, x, counts):
    """counts: int32 CUDA tensor [total atoms] (out)."""
    st = lib().ffmin_neighbour_counts(C.c_void_p(handle), C.c_void_p(x.data_ptr()),
                                      C.c_void_p(counts.data_ptr()))
    _check(st, handle)


def ffmin_mlp_work_floats():
    return int(lib().ffmin_mlp_work_floats())


def ffmin_mlp_train(feat, target, steps, batch, lr, seed, w32, adam, work, w16=None, stream=None):
    """Adam steps of the preconditioner network on the GPU (float32 CUDA
    tensors: feat [n, 5], target [n], w32 [449] in/out, adam [898] in/out,
    work [ffmin_mlp_work_floats()]; w16 optional [449] uint16/int16 out).
    Returns the per-step minibatch losses (numpy)."""
    n = int(target.numel())
    losses = np.zeros(max(steps, 1), dtype=np.float32)
    st = lib().ffmin_mlp_train(
        C.c_void_p(feat.data_ptr()), C.c_void_p(target.data_ptr()), n, int(steps), int(batch),
        float(lr), int(seed), C.c_void_p(w32.data_ptr()),
        C.c_void_p(adam.data_ptr()) if adam is not None else None, C.c_void_p(work.data_ptr()),
        losses.ctypes.data_as(C.POINTER(C.c_float)),
        C.c_void_p(w16.data_ptr()) if w16 is not None else None, C.c_void_p(_stream_handle(stream)))
    if st != FFMIN_OK:
        raise FfminError(st, "ffmin_mlp_train failed")
    return losses


def ffmin_autotune(handle, x):
    """Pick the fastest work-item layout (and FP32 tile shape) for
    coordinates x; returns the density."""
    d = C.c_int32()
    _check(lib().ffmin_autotune(C.c_void_p(handle), _dev_ptr(x, ffmin_n_atoms(handle)), C.byref(d)), handle)
    return d.value


def ffmin_set_tuning(handle, density, f32_atoms_per_thread):
    _check(lib().ffmin_set_tuning(C.c_void_p(handle), int(density), int(f32_atoms_per_thread)), handle)


def ffmin_get_tuning(handle):
    """(items per resident block, FP32 i-atoms per thread)"""
    d, s = C.c_int32(), C.c_int32()
    _check(lib().ffmin_get_tuning(C.c_void_p(handle), C.byref(d), C.byref(s)), handle)
    return d.value, s.value
