"""Seeded synthetic inputs for short-range MD: lattices, velocities, replica sets.

This module holds no force, integrator or neighbour arithmetic.  It only draws initial states,
which the CUDA library and the CPU oracle both receive unchanged.  Random numbers come from
numpy's PCG64 generator seeded with the caller's integer.

Workloads (Sec. 3.1 of the paper describes a cubic grid of atoms with random velocities; the
workloads here use an fcc lattice instead):
  * ``fcc_lattice``      4 n^3 atoms on an fcc lattice of n^3 unit cells at density rho.
  * ``cubic_lattice``    N_e^3 atoms on a simple cubic grid at density rho (the paper's initial
                         state, Sec. 3.1).
  * ``fcc_subset``       N atoms drawn without replacement from the smallest fcc lattice with
                         at least N sites, box scaled so that the density is rho.
  * ``maxwell``          Gaussian velocity components, zero net momentum, rescaled so that
                         sum m v^2 / (3 (N - 1)) equals T exactly.
  * ``perturb``          uniform displacements in [-amp, amp] per coordinate, for snapshots with
                         non-zero forces (the perfect lattice has F = 0).
  * ``replica_specs``    (N_r, rho_r) pairs drawn uniformly for batches of independent systems.
"""
from __future__ import annotations

import math

import numpy as np

_FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def box_side(n_atoms: int, rho: float) -> float:
    return (float(n_atoms) / float(rho)) ** (1.0 / 3.0)


def _fcc_sites(ncell: int, a: float) -> np.ndarray:
    """All 4 ncell^3 sites, offset by a/4 so that no site sits on a cell face."""
    g = np.arange(ncell, dtype=np.float64)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    corners = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    sites = (corners[:, None, :] + _FCC_BASIS[None, :, :]).reshape(-1, 3)
    return (sites + 0.25) * a


def fcc_lattice(ncell: int, rho: float):
    """Perfect fcc lattice of ncell^3 unit cells at density rho: (x [4 ncell^3, 3], box [3])."""
    n = 4 * ncell ** 3
    L = box_side(n, rho)
    x = _fcc_sites(ncell, L / ncell)
    x = np.mod(x, L)
    return np.ascontiguousarray(x), np.array([L, L, L])


def cubic_lattice(n_edge: int, rho: float, serpentine: bool = False):
    """Simple cubic grid of n_edge^3 atoms at density rho, offset by half a spacing: (x, box).
    serpentine: the sites ordered along a path that reverses direction in every row and plane,
    so that consecutive sites are lattice neighbours (chains of consecutive ids, bond = spacing)."""
    n = int(n_edge) ** 3
    L = box_side(n, rho)
    a = L / n_edge
    if serpentine:
        # rows alternate in x within a plane; odd planes walk the plane's path backwards
        plane = [(x if y % 2 == 0 else n_edge - 1 - x, y) for y in range(n_edge) for x in range(n_edge)]
        idx = []
        for z in range(n_edge):
            for (x, y) in (plane if z % 2 == 0 else plane[::-1]):
                idx.append((x, y, z))
        x = (np.array(idx, dtype=np.float64) + 0.5) * a
    else:
        g = (np.arange(n_edge, dtype=np.float64) + 0.5) * a
        cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
        x = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    return np.ascontiguousarray(x), np.array([L, L, L])


def fcc_subset(n_atoms: int, rho: float, seed: int):
    """N atoms on a random subset of fcc sites at density rho: (x [N, 3], box [3])."""
    n_atoms = int(n_atoms)
    ncell = max(1, int(math.ceil((n_atoms / 4.0) ** (1.0 / 3.0) - 1e-9)))
    while 4 * ncell ** 3 < n_atoms:
        ncell += 1
    L = box_side(n_atoms, rho)
    sites = _fcc_sites(ncell, L / ncell)
    if sites.shape[0] > n_atoms:
        pick = np.sort(_rng(seed).choice(sites.shape[0], size=n_atoms, replace=False))
        sites = sites[pick]
    x = np.mod(sites, L)
    return np.ascontiguousarray(x), np.array([L, L, L])


def maxwell(n_atoms: int, temperature: float, seed: int, mass: float = 1.0) -> np.ndarray:
    """Velocities [N, 3]: Gaussian, zero total momentum, exact temperature T."""
    v = _rng(seed).standard_normal((int(n_atoms), 3))
    v -= v.mean(axis=0, keepdims=True)
    if n_atoms > 1:
        t_now = mass * float(np.sum(v * v)) / (3.0 * (n_atoms - 1))
        v *= math.sqrt(temperature / t_now)
    return np.ascontiguousarray(v)


def perturb(x: np.ndarray, box: np.ndarray, amp: float, seed: int) -> np.ndarray:
    """Displace every coordinate by U(-amp, amp) and wrap back into [0, L)."""
    d = _rng(seed).uniform(-amp, amp, size=x.shape)
    y = np.mod(x + d, np.asarray(box)[None, :])
    y[y >= np.asarray(box)[None, :]] = 0.0
    return np.ascontiguousarray(y)


def replica_specs(n_rep: int, n_min: int, n_max: int, rho_min: float, rho_max: float, seed: int):
    """[(N_r, rho_r)] for n_rep independent systems, N_r ~ U{n_min..n_max}, rho_r ~ U[rho_min, rho_max]."""
    g = _rng(seed)
    ns = g.integers(n_min, n_max + 1, size=int(n_rep))
    rhos = g.uniform(rho_min, rho_max, size=int(n_rep))
    return [(int(a), float(b)) for a, b in zip(ns, rhos)]


def replica_states(specs, temperature: float, seed: int, mass: float = 1.0):
    """Initial states for a replica set: list of (x [N_r, 3], v [N_r, 3], box [3])."""
    out = []
    for r, (n, rho) in enumerate(specs):
        x, box = fcc_subset(n, rho, seed * 100003 + 2 * r)
        v = maxwell(n, temperature, seed * 100003 + 2 * r + 1, mass)
        out.append((x, v, box))
    return out
