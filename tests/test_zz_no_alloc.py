"""The allocation-free pair energy + gradient (for callers that cannot let a
library allocate device memory: applications held to another framework's
capped memory pool, or latency-bound loops that cannot afford cudaMalloc's
implicit synchronisation).  Its output, computed with the library's fixed
internal scratch array, must match the allocating path (ffmin_energy_grad on
the same system without bonded terms) within the FP64 parity tolerances,
on two calls in a row (the scratch keeps the previous call's contents).
This file is collected last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest

from paper_1810_03358_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def pair_only(s):
    t = synth.System(**{k: getattr(s, k) for k in ("x", "x_ref", "charge", "sigma", "epsilon")},
                     bond_idx=s.bond_idx[:0], bond_k=s.bond_k[:0], bond_r0=s.bond_r0[:0],
                     angle_idx=s.angle_idx[:0], angle_k=s.angle_k[:0],
                     angle_theta0=s.angle_theta0[:0], dihedral_idx=s.dihedral_idx[:0],
                     dihedral_v=s.dihedral_v[:0], coulomb_c=s.coulomb_c)
    return t


@pytest.mark.parametrize("n,seed", [(1000, 501), (129, 502), (4000, 503)])
def test_noalloc_matches_allocating_path(n, seed):
    ffmin = need_gpu()
    import torch
    s = pair_only(synth.make_system(n, seed))
    dev = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float64, device="cuda")
    x, q, sg, ep = dev(s.x), dev(s.charge), dev(s.sigma), dev(s.epsilon)
    S = ffmin.System([s], ffmin.FFMIN_FP64)
    e_ref, g_ref = S.energy_grad(x)
    S.close()
    g_ref = g_ref.cpu().numpy()
    scale_e = np.abs(e_ref[0]) + 1.0
    scale_g = np.abs(g_ref).max()
    for call in range(2):
        g = torch.full_like(x, float("nan"))
        e = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        ffmin.ffmin_pair_energy_grad_noalloc(x, q, sg, ep, g, e, coulomb_c=s.coulomb_c)
        torch.cuda.synchronize()
        assert abs(e.item() - e_ref[0]) <= 1e-11 * scale_e, (call, e.item(), e_ref[0])
        assert np.abs(g.cpu().numpy() - g_ref).max() <= 1e-9 * scale_g, call


def test_noalloc_rejects_too_many_atoms():
    ffmin = need_gpu()
    import torch
    n = 8193
    z = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    w = torch.ones(n, dtype=torch.float64, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ffmin.FfminError) as ei:
        ffmin.ffmin_pair_energy_grad_noalloc(z, w, w, w, z.clone(), e)
    assert ei.value.status == ffmin.FFMIN_ERR_INVALID_ARG
