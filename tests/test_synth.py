"""The input generator: seeded, deterministic, and its files round-trip."""
import os

import numpy as np

from paper_1810_03358_gb300 import synth


def test_generator_is_deterministic():
    a, b = synth.make_system(300, 9), synth.make_system(300, 9)
    assert synth.digest(a) == synth.digest(b)
    assert synth.digest(a) != synth.digest(synth.make_system(300, 10))


def test_paper_workload_shape():
    s = synth.make_system(500, 1)
    assert s.x.shape == (500, 3) and s.bond_idx.shape == (499, 2) and s.dihedral_idx.shape == (497, 4)
    assert abs(s.charge.sum()) < 1e-12
    assert s.sigma.min() >= 2.5 and s.sigma.max() <= 3.8
    assert s.epsilon.min() >= 0.02 and s.epsilon.max() <= 0.2
    # bonds of the reference chain are 1.5 A; the start is jittered N(0, 0.3 A)
    d = np.linalg.norm(s.x_ref[1:] - s.x_ref[:-1], axis=1)
    assert np.allclose(d, 1.5, atol=1e-9)
    assert 0.2 < np.std(s.x - s.x_ref) < 0.4


def test_npz_round_trip(tmp_path):
    s = synth.make_system(120, 4)
    path = os.path.join(tmp_path, "s.npz")
    h = synth.save_npz(s, path)
    t = synth.load_npz(path)
    assert synth.digest(t) == h == synth.digest(s)
