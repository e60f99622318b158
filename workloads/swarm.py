"""Seeded uniforms drawn by the particle swarm integer search (input only).

The swarm of Section 2.1 starts each particle at a random position with a
random velocity and draws r1, r2 in [0, 1) for every update of Eq. 2.  These
numbers are inputs to the search: both the oracle and a device search take
the same array, so that a swarm's path is reproducible across the two.  This
module only draws them; what they mean is the search's business.

Layout: ``u[k, t, i, 0:4]`` for POI k, generation t, particle i.  Generation
0 holds the start draws (two for the position, two for the velocity);
generation t >= 1 holds r1 (x, y) and r2 (x, y) of the update that produces
generation t.
"""
from __future__ import annotations

import numpy as np

PARTICLES = 50    # swarm size of Section 5
GENERATIONS = 5   # generation cap of Section 2.1 (after Wu et al.)


def uniforms(seed: int, n_poi: int, generations: int = GENERATIONS,
             particles: int = PARTICLES) -> np.ndarray:
    """float64 uniforms in [0, 1), shape (n_poi, generations, particles, 4)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5357524D, int(seed)]))
    return rng.random((n_poi, generations, particles, 4))
