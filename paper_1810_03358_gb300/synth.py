"""Seeded synthetic force-field systems (input generator only).

This module draws the inputs that both the CUDA path and the FP64 CPU oracle
consume: atom coordinates, per-atom charge / Lennard-Jones parameters and the
bonded topology of a compact self-avoiding chain.  It contains none of the
energy or minimizer arithmetic; it only places atoms and draws parameters.

The workloads stand in for the protein-protein docking poses of the paper's
experiments (Section 5.3), which are not available: a chain of N atoms with
1.5 A bonds grown inside a sphere of density 0.1 atoms/A^3 (a protein-like
globule), charges U[-0.8, 0.8] e shifted to net zero, sigma U[2.5, 3.8] A,
epsilon U[0.02, 0.2] kcal/mol, harmonic bonds (K = 300 kcal/mol/A^2,
r0 = 1.5 A), harmonic angles (K = 60 kcal/mol/rad^2, theta0 = the generated
angle), OPLS torsions with V1..V4 ~ U[0, 1] kcal/mol, and coordinates
jittered by N(0, 0.3 A) with a separate seed.  The force-field form is the
one of Section 2 (stretch, bend, torsion, Coulomb, Lennard-Jones).
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass, field

import numpy as np

# Coulomb constant in kcal*A/(mol*e^2): the paper's 1389.38757 kJ*A/(mol*e^2)
# (Section 2, Coulomb term) divided by 4.184 kJ/kcal.
COULOMB_KCAL = 1389.38757 / 4.184

BOND_LENGTH = 1.5
BOND_K = 300.0
ANGLE_K = 60.0
MIN_NONBONDED_SEP = 1.6
DENSITY = 0.1
JITTER_SIGMA = 0.3


@dataclass
class System:
    """One synthetic system; all arrays are numpy, FP64 / int32, C-contiguous."""

    x: np.ndarray            # [N, 3] jittered start coordinates (A)
    x_ref: np.ndarray        # [N, 3] unjittered chain (reference geometry)
    charge: np.ndarray       # [N] e
    sigma: np.ndarray        # [N] A
    epsilon: np.ndarray      # [N] kcal/mol
    bond_idx: np.ndarray     # [nb, 2] int32
    bond_k: np.ndarray       # [nb]
    bond_r0: np.ndarray      # [nb]
    angle_idx: np.ndarray    # [na, 3] int32, vertex in the middle
    angle_k: np.ndarray      # [na]
    angle_theta0: np.ndarray  # [na] rad
    dihedral_idx: np.ndarray  # [nd, 4] int32
    dihedral_v: np.ndarray   # [nd, 4] V1..V4
    coulomb_c: float = COULOMB_KCAL
    # 0: every pair interacts (the paper); 1: bonded and angle-end pairs
    # excluded, dihedral-end pairs scaled by scale14 (force-field variant)
    exclusions: int = 0
    scale14: float = 0.5
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.x.shape[0])


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _unit(v):
    s = 1.0 / math.sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2])
    return (v[0] * s, v[1] * s, v[2] * s)


def _place(a, b, c, length, theta, phi):
    """Place atom d from a, b, c with |cd| = length, angle bcd = theta and
    dihedral abcd = phi (natural-extension-reference-frame construction)."""
    bc = _unit(_sub(c, b))
    n = _unit(_cross(_sub(b, a), bc))
    m = _cross(n, bc)
    d0 = -length * math.cos(theta)
    d1 = length * math.sin(theta) * math.cos(phi)
    d2 = length * math.sin(theta) * math.sin(phi)
    return (c[0] + d0 * bc[0] + d1 * m[0] + d2 * n[0],
            c[1] + d0 * bc[1] + d1 * m[1] + d2 * n[1],
            c[2] + d0 * bc[2] + d1 * m[2] + d2 * n[2])


class _Cells:
    """Uniform cell grid for the self-avoidance test."""

    def __init__(self, size):
        self.size = size
        self.cells: dict[tuple, list] = {}

    def key(self, p):
        s = self.size
        return (int(math.floor(p[0] / s)), int(math.floor(p[1] / s)), int(math.floor(p[2] / s)))

    def add(self, idx, p):
        self.cells.setdefault(self.key(p), []).append(idx)

    def remove(self, idx, p):
        self.cells[self.key(p)].remove(idx)

    def clash(self, p, pos, max_idx, dmin2):
        kx, ky, kz = self.key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    lst = self.cells.get((kx + dx, ky + dy, kz + dz))
                    if not lst:
                        continue
                    for j in lst:
                        if j <= max_idx:
                            q = pos[j]
                            ex = p[0] - q[0]
                            ey = p[1] - q[1]
                            ez = p[2] - q[2]
                            if ex * ex + ey * ey + ez * ez < dmin2:
                                return True
        return False


def grow_chain(n_atoms: int, rng: np.random.Generator):
    """Self-avoiding chain inside a sphere of density DENSITY.

    Returns (positions [N,3], bond angle at each interior atom [N-2]).
    Each new atom: bond 1.5 A, bond angle U[100, 120] deg, torsion
    U[-180, 180] deg; a trial closer than 1.6 A to any atom two or more
    positions back, or outside the sphere, is rejected; after 100 rejections
    the last 5 atoms are removed and growth resumes.
    """
    if n_atoms < 1:
        raise ValueError("n_atoms must be >= 1")
    radius = (3.0 * n_atoms / (4.0 * math.pi * DENSITY)) ** (1.0 / 3.0)
    pos = [(0.0, 0.0, 0.0)] * n_atoms
    theta = [0.0] * n_atoms  # theta[k] = angle (k-2, k-1, k)
    cells = _Cells(MIN_NONBONDED_SEP)
    dmin2 = MIN_NONBONDED_SEP ** 2
    r2max = radius * radius

    # atom 0: uniform in the inner half-radius ball
    while True:
        p = tuple(float(v) for v in rng.uniform(-0.5 * radius, 0.5 * radius, size=3))
        if p[0] * p[0] + p[1] * p[1] + p[2] * p[2] <= 0.25 * r2max:
            break
    pos[0] = p
    cells.add(0, pos[0])
    k = 1
    rejects = 0
    total_trials = 0
    max_trials = 2000 * n_atoms + 100000
    while k < n_atoms:
        total_trials += 1
        if total_trials > max_trials:
            raise RuntimeError("chain growth did not finish")
        th = math.radians(float(rng.uniform(100.0, 120.0)))
        if k == 1:
            v = _unit(tuple(float(t) for t in rng.normal(size=3)))
            p = (pos[0][0] + BOND_LENGTH * v[0], pos[0][1] + BOND_LENGTH * v[1],
                 pos[0][2] + BOND_LENGTH * v[2])
        elif k == 2:
            b, c = pos[0], pos[1]
            v = tuple(float(t) for t in rng.normal(size=3))
            a = (b[0] + v[0], b[1] + v[1], b[2] + v[2])  # fixes the plane of the angle
            phi = float(rng.uniform(-math.pi, math.pi))
            p = _place(a, b, c, BOND_LENGTH, th, phi)
        else:
            phi = math.radians(float(rng.uniform(-180.0, 180.0)))
            p = _place(pos[k - 3], pos[k - 2], pos[k - 1], BOND_LENGTH, th, phi)
        ok = (p[0] * p[0] + p[1] * p[1] + p[2] * p[2] <= r2max
              and not cells.clash(p, pos, k - 2, dmin2))
        if ok:
            pos[k] = p
            theta[k] = th
            cells.add(k, p)
            k += 1
            rejects = 0
        else:
            rejects += 1
            if rejects >= 100:
                back = min(5, k - 1)
                for _ in range(back):
                    k -= 1
                    cells.remove(k, pos[k])
                rejects = 0
    return np.array(pos, dtype=np.float64), np.array(theta[2:], dtype=np.float64), radius


def make_system(n_atoms: int, seed: int, jitter_seed: int | None = None,
                torsions: bool = True) -> System:
    """Build one seeded synthetic system (chain topology, see module doc)."""
    rng = np.random.default_rng(seed)
    x_ref, theta0, radius = grow_chain(n_atoms, rng)
    q = rng.uniform(-0.8, 0.8, size=n_atoms)
    q = q - q.mean()
    sigma = rng.uniform(2.5, 3.8, size=n_atoms)
    eps = rng.uniform(0.02, 0.2, size=n_atoms)
    nb = max(n_atoms - 1, 0)
    na = max(n_atoms - 2, 0)
    nd = max(n_atoms - 3, 0)
    bonds = np.stack([np.arange(nb), np.arange(nb) + 1], axis=1).astype(np.int32)
    angles = np.stack([np.arange(na), np.arange(na) + 1, np.arange(na) + 2], axis=1).astype(np.int32)
    dih = np.stack([np.arange(nd) + i for i in range(4)], axis=1).astype(np.int32)
    vtors = rng.uniform(0.0, 1.0, size=(nd, 4))
    if not torsions:
        vtors[:] = 0.0
    jrng = np.random.default_rng(seed + 1_000_000 if jitter_seed is None else jitter_seed)
    x = x_ref + jrng.normal(0.0, JITTER_SIGMA, size=x_ref.shape)
    return System(
        x=np.ascontiguousarray(x), x_ref=np.ascontiguousarray(x_ref),
        charge=np.ascontiguousarray(q), sigma=np.ascontiguousarray(sigma),
        epsilon=np.ascontiguousarray(eps),
        bond_idx=np.ascontiguousarray(bonds.reshape(nb, 2)),
        bond_k=np.full(nb, BOND_K), bond_r0=np.full(nb, BOND_LENGTH),
        angle_idx=np.ascontiguousarray(angles.reshape(na, 3)),
        angle_k=np.full(na, ANGLE_K), angle_theta0=np.ascontiguousarray(theta0[:na]),
        dihedral_idx=np.ascontiguousarray(dih.reshape(nd, 4)),
        dihedral_v=np.ascontiguousarray(vtors.reshape(nd, 4)),
        seed=seed, meta={"radius": radius},
    )


def batch_sizes(n_sys: int = 256, seed: int = 7, lo: int = 200, hi: int = 5000) -> np.ndarray:
    """Atom counts log-uniform in [lo, hi] (the batched workload)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=n_sys)
    return np.round(np.exp(u)).astype(np.int64)


def make_batch(n_sys: int = 256, size_seed: int = 7, base_seed: int = 1000,
               lo: int = 200, hi: int = 5000) -> list[System]:
    """The batched workload: system b has N_b log-uniform atoms and seed base_seed + b."""
    sizes = batch_sizes(n_sys, size_seed, lo, hi)
    return [make_system(int(n), base_seed + b) for b, n in enumerate(sizes)]


def rigid_motion(rng: np.random.Generator):
    """A random rotation matrix and translation (for invariance tests)."""
    a = rng.normal(size=(3, 3))
    qm, r = np.linalg.qr(a)
    qm = qm * np.sign(np.diag(r))
    if np.linalg.det(qm) < 0:
        qm[:, 0] = -qm[:, 0]
    t = rng.normal(scale=5.0, size=3)
    return qm, t


_ARRAYS = ("x", "charge", "sigma", "epsilon", "bond_idx", "bond_k", "bond_r0", "angle_idx", "angle_k",
           "angle_theta0", "dihedral_idx", "dihedral_v")


def digest(s: System) -> str:
    """SHA-256 over the system's coordinates, parameters and topology (the
    exact inputs a run consumed)."""
    h = hashlib.sha256()
    for k in _ARRAYS:
        a = np.ascontiguousarray(getattr(s, k))
        h.update(k.encode())
        h.update(str(a.dtype).encode())
        h.update(str(a.shape).encode())
        h.update(a.tobytes())
    h.update(repr((float(s.coulomb_c), int(s.exclusions), float(s.scale14))).encode())
    return h.hexdigest()


def save_npz(s: System, path: str) -> str:
    """Write the system's arrays to an .npz file; returns its digest."""
    np.savez(path, **{k: getattr(s, k) for k in _ARRAYS}, coulomb_c=s.coulomb_c,
             exclusions=s.exclusions, scale14=s.scale14, seed=s.seed)
    return digest(s)


def load_npz(path: str) -> System:
    """Read a system written by save_npz."""
    d = np.load(path)
    kw = {k: d[k] for k in _ARRAYS}
    return System(x_ref=d["x"].copy(), coulomb_c=float(d["coulomb_c"]), exclusions=int(d["exclusions"]),
                  scale14=float(d["scale14"]), seed=int(d["seed"]), **kw)
