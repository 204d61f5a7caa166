"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module only draws numbers (numpy ``Generator`` streams keyed by a seed);
it holds none of the lattice Boltzmann arithmetic.  The workloads are the
paper's synthetic lattices (Sec. VI): uniform or Gaussian-perturbed densities
on a periodic box, and random populations near a given base state for the
element-by-element parity checks.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


def perturbed_density(shape, rho0: float, amplitude: float, seed: int, species: int) -> np.ndarray:
    """rho0 + amplitude * g per site, g standard normal, float64 [z][y][x]."""
    g = _rng(seed, 100 + species).standard_normal(size=tuple(shape))
    return rho0 + amplitude * g


def random_populations(base: np.ndarray, shape, rel_eps: float, seed: int) -> np.ndarray:
    """Populations base[s, i] * (1 + rel_eps * g) per site; base has shape
    [species, Q] (two species for the binary mixture, more for the N-species one).

    Returns float64 [species][Q][z][y][x] rounded to float32 values, so the same
    state is exactly representable on both sides of a parity comparison."""
    base = np.asarray(base, dtype=np.float64)
    g = _rng(seed, 200).standard_normal(size=base.shape + tuple(shape))
    f = base[:, :, None, None, None] * (1.0 + rel_eps * g)
    return f.astype(np.float32).astype(np.float64)


def batch_replica_configs(n: int, seed: int, sizes=(64, 128, 256, 512)):
    """Independent replica parameters for the batched form: nx, ny drawn from
    ``sizes``, kT log-uniform in [1e-6, 1e-4], G*rho0 uniform in [0, 0.9],
    distinct seeds.  Returns a list of dicts."""
    r = _rng(seed, 300)
    out = []
    for k in range(n):
        out.append(dict(nx=int(r.choice(sizes)), ny=int(r.choice(sizes)),
                        kT=float(10.0 ** r.uniform(-6.0, -4.0)), G=float(r.uniform(0.0, 0.9)),
                        seed=int(r.integers(1, 2**63 - 1))))
    return out
