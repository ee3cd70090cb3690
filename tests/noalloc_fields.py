"""Seeded synthetic fields for the no-allocation observables tests (inputs
only: cell codes, porosity, densities, velocities, saturation; no method
arithmetic)."""
import numpy as np


def synthetic_fields(shape, seed):
    """Random cell codes (pore, solid, gray, a few inlet and outlet cells),
    porosity, densities in [0.03, 1], velocities of order 1e-3 and saturations
    in [0, 1], as the [6][n] float32 field block lbm_get_fields writes."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    n = nx * ny * nz
    cell = np.zeros(n, np.uint8)
    r = rng.random(n)
    cell[r < 0.2] = 1
    cell[(r >= 0.2) & (r < 0.4)] = 2
    cell[(r >= 0.4) & (r < 0.41)] = 3
    cell[(r >= 0.41) & (r < 0.42)] = 4
    phi = np.where(cell == 2, 0.1 + 0.5 * rng.random(n), np.where(cell == 1, 0.0, 1.0)).astype(np.float32)
    fields = np.zeros((6, n), np.float32)
    fields[0] = 0.03 + 0.97 * rng.random(n)
    fields[1] = 1.03 - fields[0]
    fields[2:5] = 1e-3 * rng.standard_normal((3, n))
    fields[5] = rng.random(n)
    fields[:, cell == 1] = 0.0
    probe = (0.5 * (nx - 1), 0.5 * (ny - 1), 0.5 * (nz - 1), 0.2 * min(shape), 0.4 * min(shape))
    return dict(shape=shape, cell=cell, phi=phi, fields=fields, probe=probe, G=1.1)
