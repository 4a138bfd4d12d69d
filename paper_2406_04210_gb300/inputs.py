"""Seeded synthetic initial conditions for the LJ workloads.

This module is shared by the CUDA path's tests/bench and by the oracle's tests.
It holds no step of the MD method itself: only lattice placement, random
insertion, jitter and Maxwell-Boltzmann velocity draws (numpy's PCG64 through
``numpy.random.default_rng(seed)``).  The recipes follow the workloads of the
paper's truncated-force study (Sec. 5, an LJ fluid of 10^5 particles) at the
sizes of the five named configurations:

* ``lj4000``      fcc 10^3 x 4 = 4,000, rho = 0.8442, T = 0.722
* ``binary256k``  80:20 A/B mixture, 256,000 particles, rho = 1.2, T = 0.7
* ``replicas512`` 512 boxes, N log-uniform in [500, 20000], rho U[0.6, 0.95],
                  T U[0.7, 1.5]
* ``lj32000``     fcc 20^3 x 4 = 32,000, rho = 0.8442, T = 0.722
* ``lj4m``        fcc 100^3 x 4 = 4,000,000, rho = 0.8442, T = 0.722
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

#: fcc basis in units of the cubic lattice constant
_FCC = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


@dataclasses.dataclass
class System:
    """One periodic box: positions in [0, L), velocities, species ids."""

    box: np.ndarray            # (3,) float64 edge lengths
    pos: np.ndarray            # (n, 3) float64
    vel: np.ndarray            # (n, 3) float64
    type: np.ndarray           # (n,) int32
    eps: np.ndarray            # (nt, nt) float64
    sigma: np.ndarray          # (nt, nt) float64
    rcut: np.ndarray           # (nt, nt) float64
    skin: float = 0.3
    dt: float = 0.005
    T: float = 0.722
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def ntypes(self) -> int:
        return int(self.eps.shape[0])


def _wrap(pos, box):
    return pos - box * np.floor(pos / box)


def fcc_lattice(ncell: int, rho: float):
    """4 * ncell^3 fcc sites filling a cube at number density rho."""
    n = 4 * ncell ** 3
    L = (n / rho) ** (1.0 / 3.0)
    a = L / ncell
    g = np.arange(ncell, dtype=np.float64)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    pos = (cells[:, None, :] + _FCC[None, :, :]).reshape(-1, 3) * a
    return pos, np.array([L, L, L])


def jitter(pos, box, amp, rng):
    """Add a uniform displacement in [-amp, +amp] to every component."""
    return _wrap(pos + rng.uniform(-amp, amp, size=pos.shape), box)


def maxwell_boltzmann(n, T, rng):
    """Gaussian velocities (unit mass), zero net momentum, scaled so that
    sum v^2 / (3n - 3) equals T exactly."""
    v = rng.normal(0.0, math.sqrt(T), size=(n, 3))
    if n > 1:
        v -= v.mean(axis=0, keepdims=True)
        s = float(np.sum(v * v)) / (3.0 * n - 3.0)
        if s > 0:
            v *= math.sqrt(T / s)
    return v


def random_insertion(n, box, dmin, rng, batch=None):
    """Random sequential insertion of n points with pairwise minimum-image
    separation >= dmin (rejection in batches with a periodic k-d tree)."""
    from scipy.spatial import cKDTree

    box = np.asarray(box, dtype=np.float64)
    acc = np.zeros((0, 3))
    batch = batch or max(1024, n // 4)
    while acc.shape[0] < n:
        cand = rng.uniform(0.0, 1.0, size=(batch, 3)) * box
        if acc.shape[0]:
            t = cKDTree(acc, boxsize=box)
            d, _ = t.query(cand, k=1, distance_upper_bound=dmin)
            cand = cand[~np.isfinite(d) | (d >= dmin)]
        if cand.shape[0] > 1:
            tc = cKDTree(cand, boxsize=box)
            pairs = tc.query_pairs(dmin, output_type="ndarray")
            drop = np.zeros(cand.shape[0], dtype=bool)
            # greedy: keep the earlier candidate of each close pair
            for i, j in pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]:
                if not drop[i]:
                    drop[j] = True
            cand = cand[~drop]
        acc = np.concatenate([acc, cand[: n - acc.shape[0]]], axis=0)
    return acc


def _mono_params(rcut=2.5):
    return (np.ones((1, 1)), np.ones((1, 1)), np.full((1, 1), rcut))


def fcc_system(ncell, rho=0.8442, T=0.722, seed=0, jitter_amp=0.05, dt=0.005, skin=0.3,
               rcut=2.5) -> System:
    rng = np.random.default_rng(seed)
    pos, box = fcc_lattice(ncell, rho)
    pos = jitter(pos, box, jitter_amp, rng)
    vel = maxwell_boltzmann(pos.shape[0], T, rng)
    e, s, rc = _mono_params(rcut)
    return System(box, pos, vel, np.zeros(pos.shape[0], np.int32), e, s, rc, skin, dt, T, seed)


def fcc_subset_system(n, rho, T, seed, jitter_amp=0.05, dt=0.005, skin=0.3, rcut=2.5) -> System:
    """n particles on a random subset of the sites of the smallest fcc lattice
    with at least n sites, scaled to density rho, plus jitter."""
    m = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-12))
    while 4 * m ** 3 < n:
        m += 1
    rng = np.random.default_rng(seed)
    L = (n / rho) ** (1.0 / 3.0)
    g = np.arange(m, dtype=np.float64)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    sites = (cells[:, None, :] + _FCC[None, :, :]).reshape(-1, 3) * (L / m)
    pick = np.sort(rng.choice(sites.shape[0], size=n, replace=False))
    box = np.array([L, L, L])
    pos = jitter(sites[pick], box, jitter_amp, rng)
    vel = maxwell_boltzmann(n, T, rng)
    e, s, rc = _mono_params(rcut)
    return System(box, pos, vel, np.zeros(n, np.int32), e, s, rc, skin, dt, T, seed)


def binary_params():
    """80:20 A/B LJ mixture: eps_AB = 1.5, sigma_AB = 0.8, eps_BB = 0.5,
    sigma_BB = 0.88, rc_ab = 2.5 sigma_ab."""
    eps = np.array([[1.0, 1.5], [1.5, 0.5]])
    sig = np.array([[1.0, 0.8], [0.8, 0.88]])
    return eps, sig, 2.5 * sig


def binary_random_system(n=256000, rho=1.2, T=0.7, seed=0, dmin=0.7, dt=0.003,
                         skin=0.3) -> System:
    """Unrelaxed binary mixture: random insertion with minimum separation dmin
    (first 0.8 n are species A).  The workload relaxes this configuration with
    an FP64 minimiser before use."""
    rng = np.random.default_rng(seed)
    L = (n / rho) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    pos = random_insertion(n, box, dmin, rng)
    t = np.zeros(n, np.int32)
    t[int(round(0.8 * n)):] = 1
    vel = maxwell_boltzmann(n, T, rng)
    eps, sig, rc = binary_params()
    return System(box, pos, vel, t, eps, sig, rc, skin, dt, T, seed)


def replica_systems(nrep=512, nmin=500, nmax=20000, rho_range=(0.6, 0.95),
                    T_range=(0.7, 1.5), seed=0, dt=0.005, skin=0.3):
    """Independent monatomic boxes with log-uniform particle counts."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=nrep))).astype(int)
    rhos = rng.uniform(*rho_range, size=nrep)
    Ts = rng.uniform(*T_range, size=nrep)
    seeds = rng.integers(0, 2 ** 31 - 1, size=nrep)
    return [fcc_subset_system(int(n), float(r), float(t), int(s), dt=dt, skin=skin)
            for n, r, t, s in zip(ns, rhos, Ts, seeds)]


#: fixed seeds of the named workloads
SEEDS = {"lj4000": 2406042101, "binary256k": 2406042102, "replicas512": 2406042103,
         "lj32000": 2406042104, "lj4m": 2406042105}


def lj4000(seed=SEEDS["lj4000"]):
    return fcc_system(10, seed=seed)


def lj32000(seed=SEEDS["lj32000"]):
    return fcc_system(20, seed=seed)


def lj4m(seed=SEEDS["lj4m"]):
    return fcc_system(100, seed=seed)
