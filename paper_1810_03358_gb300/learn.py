"""Learned per-atom diagonal preconditioner for L-BFGS (an extension; the
paper has no learned part).

Data: plain L-BFGS trajectories run by the library itself (ffmin_minimize with
recording).  For a recorded step with s = x_{k+1} - x_k, y = g_{k+1} - g_k the
target of atom i is log((<s_i, y_i> / <y_i, y_i>) / gamma), gamma = <s, y> /
<y, y> of the whole system: how much larger (or smaller) than the global
scale the atom's own secant curvature ratio is.  Only atoms with
<s_i, y_i> > 0 count.  Features: charge, sigma, epsilon, neighbours within
8 A (of the starting structure) / 64, log(1 + |g_i|) at x_k.

Training runs on the GPU through ffmin_mlp_train (hand-written forward,
backward and Adam kernels); inference runs inside the L-BFGS direction
kernel (ffmin_set_precond + options.use_learned_precond), with plain L-BFGS
as the fallback whenever the scaled direction is not a descent direction.
"""
from __future__ import annotations

import os

import numpy as np

from . import ffmin, synth

N_PARAMS = 449


def init_weights(seed: int = 0) -> np.ndarray:
    """He-style random first layer, zero output layer (starts at d = 1)."""
    rng = np.random.default_rng(seed)
    w = np.zeros(N_PARAMS, dtype=np.float32)
    w[:320] = rng.normal(0.0, np.sqrt(2.0 / 5.0), size=320)
    return w


def record_trajectories(systems, precision=ffmin.FFMIN_MIXED, record_every=25, record_slots=40,
                        max_iter=100000):
    """Minimize the systems with plain L-BFGS, recording every record_every-th
    step; returns (features [n, 5] float32, targets [n] float32, results)."""
    import torch
    S = ffmin.System(systems, precision)
    x = torch.tensor(np.concatenate([s.x.reshape(-1) for s in systems]), dtype=torch.float64,
                     device="cuda")
    counts = torch.zeros(S.n_atoms, dtype=torch.int32, device="cuda")
    ffmin.ffmin_neighbour_counts(S.handle, x, counts)
    rec = torch.zeros(record_slots * S.n_atoms * 4, dtype=torch.float64, device="cuda")
    o = ffmin.ffmin_options_default(method="LBFGS", max_iter=max_iter, record_every=record_every,
                                    record_slots=record_slots)
    o.record_dev = rec.data_ptr()
    res = ffmin.ffmin_minimize(S.handle, x, o, S.n_sys)
    S.close()
    rec = rec.cpu().numpy().reshape(record_slots, -1, 4)
    n8 = counts.cpu().numpy()
    q = np.concatenate([s.charge for s in systems])
    sg = np.concatenate([s.sigma for s in systems])
    ep = np.concatenate([s.epsilon for s in systems])
    offs = np.cumsum([0] + [s.n_atoms for s in systems])
    feats, targs = [], []
    for slot in range(record_slots):
        r = rec[slot]
        for b in range(len(systems)):
            a0, a1 = offs[b], offs[b + 1]
            rb = r[a0:a1]
            if not np.all(rb[:, 3] == 1.0):
                continue
            sy, yy, gn = rb[:, 0], rb[:, 1], rb[:, 2]
            gamma = sy.sum() / yy.sum() if yy.sum() > 0 else 0.0
            ok = (sy > 0) & (yy > 0)
            if not gamma > 0 or not ok.any():
                continue
            t = np.log((sy[ok] / yy[ok]) / gamma)
            f = np.stack([q[a0:a1][ok], sg[a0:a1][ok], ep[a0:a1][ok], n8[a0:a1][ok] / 64.0,
                          np.log1p(gn[ok])], axis=1)
            feats.append(f)
            targs.append(t)
    if not feats:
        return np.zeros((0, 5), np.float32), np.zeros(0, np.float32), res
    return (np.concatenate(feats).astype(np.float32), np.concatenate(targs).astype(np.float32), res)


def train(feat, target, steps=400, batch=8192, lr=3e-3, seed=1, w0=None):
    """Adam on the GPU; returns (w32 float32 [449], w16 float16 [449], losses)."""
    import torch
    f = torch.tensor(np.ascontiguousarray(feat, dtype=np.float32), device="cuda")
    t = torch.tensor(np.ascontiguousarray(target, dtype=np.float32), device="cuda")
    w32 = torch.tensor(init_weights(seed) if w0 is None else w0, dtype=torch.float32, device="cuda")
    adam = torch.zeros(2 * N_PARAMS, dtype=torch.float32, device="cuda")
    work = torch.zeros(ffmin.ffmin_mlp_work_floats(), dtype=torch.float32, device="cuda")
    w16 = torch.zeros(N_PARAMS, dtype=torch.int16, device="cuda")
    losses = ffmin.ffmin_mlp_train(f, t, steps, batch, lr, seed, w32, adam, work, w16)
    w16h = w16.cpu().numpy().view(np.float16)
    return w32.cpu().numpy(), w16h, losses


def gradient(feat, target, w32):
    """Mean-loss gradient of the network over all rows (GPU kernels)."""
    import torch
    f = torch.tensor(np.ascontiguousarray(feat, dtype=np.float32), device="cuda")
    t = torch.tensor(np.ascontiguousarray(target, dtype=np.float32), device="cuda")
    w = torch.tensor(np.ascontiguousarray(w32, dtype=np.float32), device="cuda")
    work = torch.zeros(ffmin.ffmin_mlp_work_floats(), dtype=torch.float32, device="cuda")
    ffmin.ffmin_mlp_train(f, t, 0, int(t.numel()), 0.0, 0, w, None, work)
    return work[-N_PARAMS:].cpu().numpy()


def minimize_with(systems, w16, precision=ffmin.FFMIN_MIXED, use=True, max_iter=100000, **opts):
    """L-BFGS with (use=True) or without the learned diagonal (further
    ffmin options by keyword); returns results, seconds and the final x."""
    import torch
    S = ffmin.System(systems, precision)
    if w16 is not None:
        ffmin.ffmin_set_precond(S.handle, w16)
    x = torch.tensor(np.concatenate([s.x.reshape(-1) for s in systems]), dtype=torch.float64,
                     device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    res = S.minimize(x, method="LBFGS", max_iter=max_iter, use_learned_precond=1 if use else 0, **opts)
    ev1.record()
    torch.cuda.synchronize()
    S.close()
    return res, ev0.elapsed_time(ev1) / 1e3, x


def training_systems(n_sys=128, seed0=10000, lo=1000, hi=5000):
    """n_sys systems with sizes uniform in [lo, hi] (size seed seed0) and
    seeds seed0, seed0 + 1, ...; a seed whose chain growth gives up is
    skipped (the next seed takes its place)."""
    rng = np.random.default_rng(seed0)
    sizes = rng.integers(lo, hi + 1, size=n_sys)
    out, seed = [], seed0
    for n in sizes:
        while True:
            try:
                out.append(synth.make_system(int(n), seed))
                break
            except RuntimeError:
                pass
            finally:
                seed += 1
    return out


# FP16 weights written by main() (the shipped network)
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "precond_w16.npy")


def load_weights(path: str = WEIGHTS):
    """The shipped FP16 weights (449 values) or None when absent."""
    return np.load(path) if os.path.exists(path) else None


def evaluate(n_atoms=30000, seeds=(100000,), precision=ffmin.FFMIN_MIXED, max_iter=100000):
    """Held-out comparison: each seed's n_atoms system minimized by plain
    L-BFGS and by L-BFGS with the shipped network, one system at a time;
    returns one dict per seed (iterations, evaluations, seconds, energies,
    statuses of both runs)."""
    w16 = load_weights()
    if w16 is None:
        raise RuntimeError(f"{WEIGHTS} is missing: train the network first (learn.main)")
    out = []
    for seed in seeds:
        s = synth.make_system(n_atoms, seed)
        row = {"seed": seed, "n_atoms": n_atoms}
        for tag, use in (("plain", False), ("learned", True)):
            res, sec, _ = minimize_with([s], w16, precision=precision, use=use, max_iter=max_iter)
            r = res[0]
            row[tag] = {"status": r["status_name"], "iterations": r["iterations"],
                        "evals": r["energy_evals"] + r["grad_evals"], "seconds": sec,
                        "energy": r["energy"], "grad_inf": r["grad_inf"]}
        out.append(row)
    return out


def main(argv=None):
    """Train the shipped weights: plain MIXED L-BFGS trajectories of n_sys
    systems with 1,000-5,000 atoms (seeds 10000 + b), recorded every 20
    steps (40 records), 1,500 Adam steps of 16,384 samples."""
    import argparse
    import time
    ap = argparse.ArgumentParser()
    ap.add_argument("--systems", type=int, default=256)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--evaluate", type=int, default=0, metavar="N_ATOMS",
                    help="compare plain and learned L-BFGS on held-out systems of this size")
    ap.add_argument("--seeds", default="100000")
    a = ap.parse_args(argv)
    if a.evaluate:
        import json
        for row in evaluate(a.evaluate, [int(v) for v in a.seeds.split(",")]):
            print(json.dumps(row), flush=True)
        return
    t0 = time.time()
    systems = training_systems(n_sys=a.systems, seed0=10000, lo=1000, hi=5000)
    t1 = time.time()
    feat, targ, _ = record_trajectories(systems, record_every=20, record_slots=40)
    t2 = time.time()
    w32, w16, losses = train(feat, targ, steps=a.steps, batch=16384, lr=3e-3, seed=3)
    t3 = time.time()
    np.save(a.out, w16)
    print(f"systems={a.systems} samples={len(targ)} target_var={targ.var():.4f} "
          f"loss first={losses[:5].mean():.4f} last={losses[-50:].mean():.4f} "
          f"gen={t1 - t0:.1f}s record={t2 - t1:.1f}s train={t3 - t2:.1f}s -> {a.out}")


if __name__ == "__main__":
    main()
