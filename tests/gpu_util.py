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
