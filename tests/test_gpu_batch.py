"""Parity of the large-batch path with the FP64 oracle, through the C ABI.

From 8 systems up, a batch takes its own reduction and control path: one
block per system sums that system's tile partials (k_sysreduce) and runs its
control step, instead of the last block of each per-tile kernel.  The
256-system workload (atom counts log-uniform in [200, 5000]) runs exactly
this path, so it is compared here with the oracle system by system on
batches of 16, 64 and 256 systems drawn from that workload's generator
(sizes capped where the oracle's minimizations would take too long).

Bars are those of the single-system tests: FP64 energy within 2e-11 of
sum|terms| and gradient within 1e-9 of the largest force; MIXED energy
within 1e-5 of sum|terms| plus the first-order effect of the FP32 position
rounding (tests.gpu_util.mixed_position_bound: 12 * 2 sqrt(3) u |x|max /
r_min, up to 1.8e-4 at the batch's closest jittered pairs, 0.29 A) and
gradient within 1e-4 of the largest force;
L-BFGS prefixes of 60 accepted steps with the oracle's exact iteration and
evaluation counts (test_gpu_minimize.prefix_parity)."""
import numpy as np
import pytest

from paper_1810_03358_gb300 import synth
from tests.gpu_util import (_oracle_energy_terms, _oracle_minimize, mixed_position_bound, need_gpu, oracle_map,
                            split, to_dev)
from tests.test_gpu_minimize import PREFIX, PREFIX_FGM, prefix_parity

pytestmark = pytest.mark.gpu

TOL = {0: dict(e=2e-11, g=1e-9), 1: dict(e=1e-5, g=1e-4)}


@pytest.fixture(scope="module")
def ff():
    return need_gpu()


def batch_systems(n_sys, cap):
    """The first n_sys systems of the 256-system workload (system b: seed
    1000 + b, size from the log-uniform draw of seed 7) whose size is at most
    cap atoms."""
    sizes = synth.batch_sizes(256)
    picked = [b for b in range(256) if sizes[b] <= cap][:n_sys]
    assert len(picked) == n_sys
    return [synth.make_system(int(sizes[b]), 1000 + b) for b in picked]


def energy_parity(ffmin, systems, prec):
    S = ffmin.System(systems, prec)
    x = to_dev([s.x for s in systems])
    e, g = S.energy_grad(x)
    e_only = S.energy(x)
    S.close()
    g = split(g.cpu().numpy(), systems)
    ref = oracle_map(_oracle_energy_terms, systems, [s.x for s in systems])
    worst_e = worst_g = 0.0
    for b, (d, st, go) in enumerate(ref):
        assert st == 0
        err_e = abs(e[b] - d["total"]) / d["sum_abs"]
        err_g = np.abs(g[b] - go).max() / np.abs(go).max()
        bar_e = TOL[prec]["e"] + (mixed_position_bound(systems[b].x) if prec == 1 else 0.0)
        assert err_e <= bar_e, (b, err_e, bar_e)
        assert err_g <= TOL[prec]["g"], (b, err_g)
        assert abs(e_only[b] - e[b]) <= 2 * bar_e * d["sum_abs"], b
        worst_e, worst_g = max(worst_e, err_e), max(worst_g, err_g)
    return worst_e, worst_g


@pytest.mark.parametrize("n_sys,cap", [(16, 1500), (64, 1500)])
def test_batch_energy_grad_fp64(ff, n_sys, cap):
    energy_parity(ff, batch_systems(n_sys, cap), 0)


def test_batch256_energy_grad_mixed(ff):
    # the full 256-system workload at its jittered start, MIXED precision
    e, g = energy_parity(ff, synth.make_batch(256), 1)
    print(f"batch256 MIXED vs oracle: energy {e:.2e} of sum|terms|, gradient {g:.2e} of max force")


@pytest.mark.parametrize("n_sys,cap", [(16, 1500), (64, 700)])
def test_batch_lbfgs_prefix_fp64(ff, oracle_mod, n_sys, cap):
    # every system of the batch takes the oracle's own steps: same counts,
    # energies within 1e-8, coordinates within 1e-6 A after 60 steps
    systems = batch_systems(n_sys, cap)
    kw = dict(method=3, lbfgs_m=10, max_iter=PREFIX)
    S = ff.System(systems, 0)
    x = to_dev([s.x for s in systems])
    rg = S.minimize(x, **kw)
    S.close()
    xg = split(x.cpu().numpy(), systems)
    ref = oracle_map(_oracle_minimize, systems, [s.x for s in systems], [kw] * n_sys)
    for b, s in enumerate(systems):
        prefix_parity(oracle_mod, s, xg[b], rg[b], kw, ref=ref[b])
        assert rg[b]["fp64_iterations"] == rg[b]["iterations"], b  # FP64 pair terms throughout


def test_batch_other_methods_prefix_fp64(ff, oracle_mod):
    # the per-system control path of the other methods at n_sys >= 8
    systems = batch_systems(12, 600)
    for method in (0, 1, 2, 5):
        kw = dict(method=method, max_iter=PREFIX_FGM if method == 1 else PREFIX)
        S = ff.System(systems, 0)
        x = to_dev([s.x for s in systems])
        rg = S.minimize(x, **kw)
        S.close()
        xg = split(x.cpu().numpy(), systems)
        ref = oracle_map(_oracle_minimize, systems, [s.x for s in systems], [kw] * len(systems))
        for b, s in enumerate(systems):
            prefix_parity(oracle_mod, s, xg[b], rg[b], kw, ref=ref[b])


@pytest.mark.parametrize("ipt", [1, 2])
def test_batch_mixed_minimization_certified(ff, oracle_mod, ipt):
    # 16 systems minimized together in MIXED precision, with either FP32 tile
    # shape: every result is a valid stop of the method (the oracle's
    # gradient of the returned point below 0.1) and reports that point's
    # FP64 energy
    systems = batch_systems(16, 1500)
    S = ff.System(systems, 1)
    S.set_tuning(10, ipt)
    x = to_dev([s.x for s in systems])
    rg = S.minimize(x, method=3, max_iter=100000)
    S.close()
    xg = split(x.cpu().numpy(), systems)
    ref = oracle_map(_oracle_energy_terms, systems, xg)
    for b, (d, st, go) in enumerate(ref):
        assert rg[b]["status_name"] == "ok", (b, rg[b])
        assert np.abs(go).max() < 0.1 * (1 + 1e-6), b
        assert abs(d["total"] - rg[b]["energy"]) <= 1e-9 * abs(d["total"]), b
        assert 0 <= rg[b]["fp64_iterations"] <= rg[b]["iterations"], b  # the FP64 phase's share
    print("FP64-phase steps per system:", [r["fp64_iterations"] for r in rg])
