"""Helpers shared by the GPU parity tests."""
import numpy as np


def need_gpu():
    import pytest
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_03358_gb300 import build
    build.build()
    from paper_1810_03358_gb300 import ffmin
    ffmin.lib()
    return ffmin


def to_dev(xs):
    import torch
    flat = np.concatenate([np.asarray(x, dtype=np.float64).reshape(-1) for x in xs])
    return torch.tensor(flat, dtype=torch.float64, device="cuda")


def split(arr, systems):
    out, k = [], 0
    for s in systems:
        n = 3 * s.n_atoms
        out.append(np.asarray(arr[k:k + n]).reshape(-1, 3))
        k += n
    return out


# ---- oracle runs in worker processes (spawned, never forked after CUDA) ----
def _oracle_energy_terms(s, x):
    from oracle import oracle
    d, st, g = oracle.energy_terms(s, x, grad=True)
    return d, st, g


def _oracle_minimize(s, x, kw):
    from oracle import oracle
    return oracle.minimize(s, x, **kw)


def oracle_pool(workers=None):
    """A process pool for independent oracle calls (one per system of a
    batch), started with 'spawn' so that no worker inherits a CUDA context."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    n = workers or max(1, min(16, os.cpu_count() or 1))
    return cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))


def oracle_map(fn, *iterables):
    """fn over the arguments in worker processes; results in order."""
    with oracle_pool() as pool:
        return list(pool.map(fn, *iterables))


def _oracle_delta_rows(s, x, xp, i0, i1):
    from oracle import oracle
    return oracle.energy_delta(s, x, xp, rows=(i0, i1))


def oracle_energy_delta(s, x, xp, blocks=64):
    """The oracle's term-by-term E(xp) - E(x) and sum |term differences|, its
    pair rows split into blocks of about equal pair counts over the pool."""
    n = s.n_atoms
    cuts = sorted({int(round(n * (1.0 - np.sqrt(1.0 - k / blocks)))) for k in range(blocks + 1)})
    lo, hi = cuts[:-1], cuts[1:]
    parts = oracle_map(_oracle_delta_rows, [s] * len(lo), [x] * len(lo), [xp] * len(lo), lo, hi)
    assert all(p[2] == 0 for p in parts)
    return sum(p[0] for p in parts), sum(p[1] for p in parts)


U32 = 2.0 ** -24  # FP32 unit roundoff


def mixed_position_bound(x):
    """First-order bound, relative to the terms themselves, of what the FP32
    rounding of the positions (u |x| per coordinate, so at most
    2 sqrt(3) u |x|max on a separation) does to a pair term through its
    r^-12 power: 12 * 2 sqrt(3) u |x|max / r_min, r_min the smallest
    separation of the configuration."""
    from scipy.spatial import cKDTree
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    if x.shape[0] < 2:
        return 0.0
    d, _ = cKDTree(x).query(x, k=2)
    return 12.0 * 2.0 * np.sqrt(3.0) * U32 * np.abs(x).max() / d[:, 1].min()
