"""Seeded inputs of the stored brute-force cases (geometry and random Fourier
tables only, no method arithmetic): a 4 bohr square cell, the first shell of
plane waves (5 G-vectors), random Hermitian-consistent slice potentials and
V = 0 electrodes."""
import math

import numpy as np

from synthetic import explicit_tables, random_tables

# (seed, E in Ry, k_par in 1/bohr, slices)
CASES = [
    (5, 3.1, (0.21, -0.13), 4),
    (6, 1.2, (0.05, 0.4), 4),
    (7, 4.0, (-0.3, 0.0), 4),
    (11, 2.6, (0.12, 0.31), 6),
    (12, 0.9, (-0.02, 0.07), 3),
]


def tiny_instance(seed, E, k, nsl):
    """The instance of one case, and its slice thicknesses."""
    rng = np.random.default_rng(seed)
    a = 4.0
    b = 2 * math.pi / a
    half = (2, 2)
    tabs = random_tables(rng, nsl, half, 0.45)
    dz = rng.uniform(0.2, 0.7, nsl)
    z = np.concatenate([[0.0], np.cumsum(dz)])
    inst = explicit_tables([a, 0.0], [0.0, a], b * b * (1 + 1e-9), z, tabs, None, None, half, [E], [k])
    return inst, dz
