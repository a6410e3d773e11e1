"""The allocation-free pair energy + gradient, for callers that cannot let a
library allocate device memory: applications held to another framework's
capped memory pool, or latency-bound loops that cannot afford cudaMalloc's
implicit synchronisation.  It computes with the library's fixed internal
scratch array; its output must match the allocating path (ffmin_energy_grad
on the same system without bonded terms) and the FP64 oracle within the FP64
parity tolerances, on two calls in a row (the scratch keeps the previous
call's contents), on the legacy stream and on a side stream.  This file is
collected last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

from paper_1810_03358_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

TOL_E, TOL_G = 2e-11, 1e-9  # of sum|terms| and of the largest force (FP64 path)


def pair_only(s):
    t = synth.System(**{k: getattr(s, k) for k in ("x", "x_ref", "charge", "sigma", "epsilon")},
                     bond_idx=s.bond_idx[:0], bond_k=s.bond_k[:0], bond_r0=s.bond_r0[:0],
                     angle_idx=s.angle_idx[:0], angle_k=s.angle_k[:0],
                     angle_theta0=s.angle_theta0[:0], dihedral_idx=s.dihedral_idx[:0],
                     dihedral_v=s.dihedral_v[:0], coulomb_c=s.coulomb_c)
    return t


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n,seed", [(1, 504), (5, 505), (129, 502), (1000, 501), (4000, 503),
                                    (8192, 506)])
def test_noalloc_matches_allocating_path_and_oracle(oracle_mod, n, seed):
    ffmin = need_gpu()
    import torch
    s = pair_only(synth.make_system(n, seed))
    x, q, sg, ep = dev(s.x), dev(s.charge), dev(s.sigma), dev(s.epsilon)
    S = ffmin.System([s], ffmin.FFMIN_FP64)
    e_ref, g_ref = S.energy_grad(x)
    S.close()
    g_ref = g_ref.cpu().numpy()
    d, st, go = oracle_mod.energy_terms(s, s.x, grad=True)
    assert st == 0
    scale_e = max(d["sum_abs"], 1e-300)
    scale_g = max(np.abs(go).max(), 1e-300)
    side = torch.cuda.Stream()
    for call, stream in enumerate([None, None, side]):
        g = torch.full_like(x, float("nan"))
        e = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ffmin.ffmin_pair_energy_grad_noalloc(x, q, sg, ep, g, e, coulomb_c=s.coulomb_c, stream=stream)
        torch.cuda.synchronize()
        ev, gv = e.item(), g.cpu().numpy()
        assert abs(ev - e_ref[0]) <= TOL_E * scale_e, (call, ev, e_ref[0])
        assert np.abs(gv - g_ref).max() <= TOL_G * scale_g, call
        assert abs(ev - d["total"]) <= TOL_E * scale_e, (call, ev, d["total"])
        assert np.abs(gv.reshape(-1, 3) - go).max() <= TOL_G * scale_g, call


def test_noalloc_reports_coincident_atoms():
    ffmin = need_gpu()
    import torch
    s = pair_only(synth.make_system(300, 507))
    xb = s.x.copy()
    xb[17] = xb[250]
    q, sg, ep = dev(s.charge), dev(s.sigma), dev(s.epsilon)
    g = torch.zeros(3 * 300, dtype=torch.float64, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ffmin.FfminError) as ei:
        ffmin.ffmin_pair_energy_grad_noalloc(dev(xb), q, sg, ep, g, e, coulomb_c=s.coulomb_c)
    assert ei.value.status == ffmin.FFMIN_ERR_NONFINITE
    # the next call on good coordinates is clean again (the flag is cleared)
    ffmin.ffmin_pair_energy_grad_noalloc(dev(s.x), q, sg, ep, g, e, coulomb_c=s.coulomb_c)
    assert np.isfinite(e.item())


def test_noalloc_rejects_bad_arguments():
    ffmin = need_gpu()
    import torch
    n = 8193
    z = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    w = torch.ones(n, dtype=torch.float64, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ffmin.FfminError) as ei:
        ffmin.ffmin_pair_energy_grad_noalloc(z, w, w, w, z.clone(), e)
    assert ei.value.status == ffmin.FFMIN_ERR_INVALID_ARG
    n = 10
    x = torch.arange(3 * n, dtype=torch.float64, device="cuda")
    w = torch.ones(n, dtype=torch.float64, device="cuda")
    for bad in (dict(coulomb_c=-1.0), dict(coulomb_c=float("nan"))):
        with pytest.raises(ffmin.FfminError) as ei:
            ffmin.ffmin_pair_energy_grad_noalloc(x, w, w, w, x.clone(), e, **bad)
        assert ei.value.status == ffmin.FFMIN_ERR_INVALID_ARG
    # buffers that do not match n are refused before any launch
    for args in ((x[:-3], w, w, w, x.clone(), e), (x, w, w, w, x[:-1].clone(), e),
                 (x.float(), w, w, w, x.clone(), e), (x, w.cpu(), w, w, x.clone(), e)):
        with pytest.raises(ffmin.FfminError) as ei:
            ffmin.ffmin_pair_energy_grad_noalloc(*args)
        assert ei.value.status == ffmin.FFMIN_ERR_INVALID_ARG
