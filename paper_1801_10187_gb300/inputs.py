"""Seeded synthetic inputs for SRD runs: the only module both the GPU path and
the CPU oracle's tests draw from.  It holds no arithmetic of the method itself.

Recipe (arXiv:1801.10187, Sec. 4 benchmark set-up and Sec. 4.1):
  * solvent positions i.i.d. uniform in the box [0, n_x) x [0, n_y) x [0, n_z)
    (cell edge a = 1), exactly ``density`` particles per cell on average
    (N = density * n_x n_y n_z);
  * velocities i.i.d. Gaussian with variance kT/m per component, then the mean
    is subtracted in double precision (Sec. 4.1: a constant correction per
    particle removes the net momentum); for the mixed-precision model the
    corrected values are rounded to float afterwards, which leaves the small
    residual the paper reports;
  * solute: linear chains grown as random walks of step r0 from a uniform
    start, wrapped into the box, Gaussian velocities with variance kT/M minus
    their own mean.
Everything is drawn from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Solvent:
    pos: np.ndarray  # (N, 3) float64 (float32-representable for mixed precision)
    vel: np.ndarray  # (N, 3) float64


def _below(L: float, dtype) -> float:
    return float(np.nextafter(dtype(L), dtype(0)))


def solvent(n_cells, density: float, kT: float = 1.0, mass: float = 1.0, seed: int = 1,
            mixed: bool = False, n_particles: int | None = None) -> Solvent:
    """Uniform positions and zero-momentum Maxwell-Boltzmann velocities."""
    nx, ny, nz = (int(x) for x in n_cells)
    N = int(round(density * nx * ny * nz)) if n_particles is None else int(n_particles)
    rng = np.random.default_rng(seed)
    L = np.array([nx, ny, nz], dtype=np.float64)
    pos = rng.random((N, 3)) * L
    vel = rng.standard_normal((N, 3)) * np.sqrt(kT / mass)
    if N > 0:
        vel -= vel.mean(axis=0)
    if mixed:
        pos = pos.astype(np.float32)
        for k in range(3):
            over = pos[:, k] >= np.float32(L[k])
            pos[over, k] = _below(L[k], np.float32)
        pos = pos.astype(np.float64)
        vel = vel.astype(np.float32).astype(np.float64)
    else:
        for k in range(3):
            over = pos[:, k] >= L[k]
            pos[over, k] = _below(L[k], np.float64)
    return Solvent(np.ascontiguousarray(pos), np.ascontiguousarray(vel))


def chains(n_cells, n_chains: int, chain_len: int, r0: float, kT: float = 1.0,
           bead_mass: float = 5.0, seed: int = 3):
    """Random-walk chains (bond length r0) wrapped into the periodic box."""
    rng = np.random.default_rng(seed)
    L = np.array([int(x) for x in n_cells], dtype=np.float64)
    nb = n_chains * chain_len
    pos = np.zeros((nb, 3))
    for c in range(n_chains):
        start = rng.random(3) * L
        steps = rng.standard_normal((chain_len - 1, 3))
        steps /= np.linalg.norm(steps, axis=1, keepdims=True)
        walk = np.vstack([start, start + np.cumsum(steps * r0, axis=0)])
        pos[c * chain_len:(c + 1) * chain_len] = walk
    pos = np.mod(pos, L)
    for k in range(3):
        over = pos[:, k] >= L[k]
        pos[over, k] = _below(L[k], np.float64)
    vel = rng.standard_normal((nb, 3)) * np.sqrt(kT / bead_mass)
    if nb > 0:
        vel -= vel.mean(axis=0)
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel)


def ensemble(n_boxes: int = 64, seed: int = 4) -> list:
    """Batched-ensemble recipe: independent periodic cubic boxes, edge L
    uniform in {16, ..., 96} cells, density 5 or 10 per cell, rotation angle
    90, 120 or 130 degrees, box seed 1000 + i; all drawn from
    ``numpy.random.default_rng(seed)``.  Initial states are thermal (drawn on
    the device from each box's seed)."""
    rng = np.random.default_rng(seed)
    edges = rng.integers(16, 97, n_boxes)
    dens = rng.choice([5, 10], n_boxes)
    angles = rng.choice([90.0, 120.0, 130.0], n_boxes)
    return [dict(n=(int(e), int(e), int(e)), density=int(d), alpha_deg=float(a), seed=1000 + i)
            for i, (e, d, a) in enumerate(zip(edges, dens, angles))]


# Named workloads (sizes of the benchmark set-ups).  Each entry gives the
# keyword arguments of the SRD parameters and of the solvent generator.
WORKLOADS = {
    "srd-10c-rho5-fp64": dict(n=(10, 10, 10), density=5, alpha_deg=130.0, dt=0.1, kT=1.0,
                              seed=1, thermostat=False, precision="fp64", steps=1000),
    "srd-100c-rho10-fp64": dict(n=(100, 100, 100), density=10, alpha_deg=130.0, dt=0.1,
                                kT=1.0, seed=2, thermostat=False, precision="fp64", steps=2000),
    "srd-100c-rho10-mixed": dict(n=(100, 100, 100), density=10, alpha_deg=130.0, dt=0.1,
                                 kT=1.0, seed=2, thermostat=False, precision="mixed",
                                 steps=2000),
    # the benchmark fluid with the Andersen-thermostat collision rule (Eq. at)
    "srd-100c-rho10-mixed-at": dict(n=(100, 100, 100), density=10, alpha_deg=130.0, dt=0.1,
                                    kT=1.0, seed=2, thermostat=False, precision="mixed",
                                    steps=2000, collision="at"),
    # the benchmark fluid with angular-momentum conservation
    "srd-100c-rho10-mixed-angular": dict(n=(100, 100, 100), density=10, alpha_deg=130.0,
                                         dt=0.1, kT=1.0, seed=2, thermostat=False,
                                         precision="mixed", steps=2000, angular=True),
    # the benchmark fluid at 8 * 10^7 particles (a 50M+ particle box)
    "srd-200c-rho10-mixed": dict(n=(200, 200, 200), density=10, alpha_deg=130.0, dt=0.1,
                                 kT=1.0, seed=4, thermostat=False, precision="mixed",
                                 steps=500),
    "srd-250c-rho5-mixed-solute": dict(n=(250, 250, 250), density=5, alpha_deg=130.0, dt=0.1,
                                       kT=1.0, seed=3, thermostat=True, precision="mixed",
                                       steps=500, n_chains=2000, chain_len=50,
                                       bead_mass=5.0, bond_k=1000.0, bond_r0=0.5,
                                       md_substeps=10),
    # the paper's polymer benchmark (Sec. 4.3): L = 50, 1024 chains of 50 beads
    # in the density-10 FP64 solvent, velocity Verlet every 0.002 (50 substeps
    # per collision), non-bonded WCA repulsion (eps = kT, sigma = 0.5)
    "srd-50c-rho10-fp64-polymer": dict(n=(50, 50, 50), density=10, alpha_deg=130.0, dt=0.1,
                                       kT=1.0, seed=5, thermostat=False, precision="fp64",
                                       steps=200, n_chains=1024, chain_len=50, bead_mass=5.0,
                                       bond_k=1000.0, bond_r0=0.5, md_substeps=50,
                                       lj_epsilon=1.0, lj_sigma=0.5),
    # the solute + thermostat workload at 1/16 of its volume (5 * 10^6 particles,
    # 128 chains): the same kernels on a state small enough to profile in full
    "srd-100c-rho5-mixed-solute": dict(n=(100, 100, 100), density=5, alpha_deg=130.0, dt=0.1,
                                       kT=1.0, seed=3, thermostat=True, precision="mixed",
                                       steps=500, n_chains=128, chain_len=50,
                                       bead_mass=5.0, bond_k=1000.0, bond_r0=0.5,
                                       md_substeps=10),
    # 64 boxes of ensemble() stepped together, against the same boxes stepped
    # one after another
    "srd-batch64-mixed": dict(kind="batch", n_boxes=64, ensemble_seed=4, dt=0.1, kT=1.0,
                              thermostat=False, precision="mixed", steps=1000),
    # Poisson arrivals of SRD jobs served by continuous batching
    "srd-served-poisson": dict(kind="serve", n_jobs=2000, rate=20.0, jobs_seed=5, l_min=10,
                               l_max=160, density=5.0, steps_min=100, steps_max=5000,
                               alpha_deg=130.0, precision="mixed", sweep_rates=(5.0, 10.0, 15.0),
                               sweep_jobs=300),
}


def avoiding_chains(n_cells, n_chains: int, chain_len: int, r0: float, min_dist: float,
                    kT: float = 1.0, bead_mass: float = 5.0, seed: int = 3):
    """Random-walk chains (bond length r0) in which no two beads, of the same
    chain or of different chains, start closer than min_dist (minimum image):
    an initial state for beads with a non-bonded repulsion.  Each step draws
    up to 200 directions; a chain that gets stuck restarts elsewhere (at most
    10^4 times, then ValueError)."""
    rng = np.random.default_rng(seed)
    L = np.array([int(x) for x in n_cells], dtype=np.float64)
    grid = {}
    placed = []

    def key(p):
        return tuple(int(x) for x in np.floor(p / 1.0) % L)

    def free(p):
        k = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    kk = ((k[0] + dx) % int(L[0]), (k[1] + dy) % int(L[1]), (k[2] + dz) % int(L[2]))
                    for q in grid.get(kk, ()):
                        d = q - p
                        d -= L * np.rint(d / L)
                        if d @ d < min_dist * min_dist:
                            return False
        return True

    for c in range(n_chains):
        for _restart in range(10000):
            chain = []
            p = rng.random(3) * L
            if not free(p):
                continue
            chain.append(p)
            ok = True
            for _ in range(chain_len - 1):
                for _try in range(200):
                    step = rng.standard_normal(3)
                    q = np.mod(chain[-1] + r0 * step / np.linalg.norm(step), L)
                    if free(q) and all(np.sum(((q - x) - L * np.rint((q - x) / L)) ** 2)
                                       >= min_dist * min_dist for x in chain):
                        break
                else:
                    ok = False
                    break
                chain.append(q)
            if ok:
                break
        else:
            raise ValueError("avoiding_chains: no room for another chain at this min_dist")
        for p in chain:
            grid.setdefault(key(p), []).append(p)
            placed.append(p)
    pos = np.array(placed).reshape(-1, 3)
    for k in range(3):
        over = pos[:, k] >= L[k]
        pos[over, k] = _below(L[k], np.float64)
    nb = n_chains * chain_len
    vel = rng.standard_normal((nb, 3)) * np.sqrt(kT / bead_mass)
    if nb > 0:
        vel -= vel.mean(axis=0)
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel)
