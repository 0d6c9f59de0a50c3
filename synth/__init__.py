"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests
and the benchmark.

This module holds no arithmetic of the particle-in-cell method: it only draws
seeded random positions, momenta and fields (numpy ``default_rng``) and
describes the workloads by their sizes.  Both sides of every parity test take
their inputs from here; neither side's arithmetic is reachable from here.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class SpeciesSpec:
    q_over_e: float
    m_over_me: float


PAIR = (SpeciesSpec(-1.0, 1.0), SpeciesSpec(+1.0, 1.0))


def grid_shape(ndim, nx, ny, nz):
    return (1 if ndim == 2 else nz, ny, nx)


def positions(rng, ndim, nx, ny, nz, n):
    """Uniform positions in the periodic box, (3, n) float64 (z = 0 in 2D)."""
    pos = np.zeros((3, n))
    pos[0] = rng.uniform(0.0, nx, n)
    pos[1] = rng.uniform(0.0, ny, n)
    if ndim == 3:
        pos[2] = rng.uniform(0.0, nz, n)
    # keep every coordinate strictly inside [0, n)
    for a, L in enumerate((nx, ny, nz)[:ndim]):
        pos[a] = np.where(pos[a] >= L, 0.0, pos[a])
    return pos


def momenta(rng, n, spread, drift=(0.0, 0.0, 0.0)):
    """Gaussian momenta u = gamma v / c with the given spread and drift, (3, n)."""
    u = rng.normal(0.0, spread, (3, n))
    for a in range(3):
        u[a] += drift[a]
    return u


def fields(rng, ndim, nx, ny, nz, amp_e, amp_b):
    """Random e and b blocks of shape (3, nz, ny, nx)."""
    shp = (3,) + grid_shape(ndim, nx, ny, nz)
    return rng.normal(0.0, amp_e, shp), rng.normal(0.0, amp_b, shp)


def random_state_arrays(seed, ndim, nx, ny, nz, ppc, spread=0.3, amp_e=0.0, amp_b=0.0,
                        species=PAIR, colocate=True):
    """Seeded raw arrays for a state: dict with e, b and a list of species dicts
    (pos, u, q_over_e, m_over_me).  With ``colocate`` every species shares the
    positions of the first one (pairs loaded on top of each other, rho = 0)."""
    rng = np.random.default_rng(seed)
    ncell = nx * ny * (1 if ndim == 2 else nz)
    n = int(round(ppc * ncell))
    e, b = fields(rng, ndim, nx, ny, nz, amp_e, amp_b)
    out = {"e": e, "b": b, "species": []}
    pos0 = positions(rng, ndim, nx, ny, nz, n)
    for k, sp in enumerate(species):
        pos = pos0.copy() if (colocate or k == 0) else positions(rng, ndim, nx, ny, nz, n)
        u = momenta(rng, n, spread)
        out["species"].append({"pos": pos, "u": u, "q_over_e": sp.q_over_e, "m_over_me": sp.m_over_me})
    return out


# Workloads of the benchmark and of the parity tests, by their sizes.
THERMAL_2D_64 = dict(name="2D3V thermal pair plasma 64x64, 16 ppc/species, theta=0.1",
                     ndim=2, nx=64, ny=64, nz=1, ppc=16, theta=0.1, n_x=0.1 ** -0.5,
                     rho_sp0=32.0, dt=0.5, steps=300, seed=1)
THERMAL_3D_128 = dict(name="3D3V thermal pair plasma 128^3, 32 ppc/species, theta=1",
                      ndim=3, nx=128, ny=128, nz=128, ppc=32, theta=1.0, n_x=1.0,
                      rho_sp0=64.0, dt=0.5, steps=1000, seed=2)
FILAMENTATION_2D_1024 = dict(name="2D3V filamentation 1024^2, 50 ppc/species, Gamma0=3 beams",
                             ndim=2, nx=1024, ny=1024, nz=1, ppc=50, theta=0.01, n_x=20.0,
                             rho_sp0=100.0, dt=0.5, steps=2000, seed=3)
