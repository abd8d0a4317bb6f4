"""Seeded synthetic lens fields (positions and masses), shared by the tests,
the benchmark and the oracle checks.

This module holds none of the ray-shooting arithmetic: it only draws numbers.
Callers pass the region to fill and, if they want a given surface density, the
total mass to rescale to.  Random draws come from numpy's PCG64 generator with
an explicit seed, so both sides of every comparison see identical inputs.

Mass shapes (the paper's flow chart "Generate lenses" and its figure captions):
  equal     all masses 1
  uniform   m ~ U[m_min, m_max]
  salpeter  dN/dm proportional to m^-2.35 on [m_min, m_max] (inverse-CDF draw)
"""
import numpy as np

SALPETER_SLOPE = 2.35


def positions_box(n, x0, x1, y0, y1, seed):
    """n positions uniform in [x0, x1) x [y0, y1), as an (n, 2) float64 array."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random((n, 2))
    xy = np.empty((n, 2))
    xy[:, 0] = x0 + (x1 - x0) * u[:, 0]
    xy[:, 1] = y0 + (y1 - y0) * u[:, 1]
    # guard the half-open upper edge against rounding up onto x1 / y1
    np.minimum(xy[:, 0], np.nextafter(x1, x0), out=xy[:, 0])
    np.minimum(xy[:, 1], np.nextafter(y1, y0), out=xy[:, 1])
    return xy


def positions_disc(n, cx, cy, r, seed):
    """n positions uniform in the disc of radius r about (cx, cy)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random((n, 2))
    rad = r * np.sqrt(u[:, 0])
    phi = 2.0 * np.pi * u[:, 1]
    return np.stack([cx + rad * np.cos(phi), cy + rad * np.sin(phi)], axis=1)


def masses(n, shape="equal", m_min=0.1, m_max=1.0, seed=0):
    """n masses of the given shape (see module docstring)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED))
    if shape == "equal":
        return np.ones(n)
    u = rng.random(n)
    if shape == "uniform":
        return m_min + (m_max - m_min) * u
    if shape == "salpeter":
        e = 1.0 - SALPETER_SLOPE
        lo, hi = m_min ** e, m_max ** e
        return (lo + (hi - lo) * u) ** (1.0 / e)
    raise ValueError(f"unknown mass shape {shape!r}")


def rescale(mass, total):
    """Scale masses by one common factor so that they sum to `total`."""
    s = float(np.sum(mass))
    if s <= 0:
        return mass.copy()
    return mass * (total / s)


def lens_field(n, box, shape="equal", m_min=0.1, m_max=1.0, seed=0, total_mass=None,
               disc=None):
    """A full field: positions in `box` = (x0, x1, y0, y1) (or in `disc` =
    (cx, cy, r) when given), masses of `shape`, optionally rescaled to
    `total_mass`.  Returns (xy (n, 2), m (n,)) float64."""
    if disc is not None:
        xy = positions_disc(n, disc[0], disc[1], disc[2], seed)
    else:
        xy = positions_box(n, box[0], box[1], box[2], box[3], seed)
    m = masses(n, shape, m_min, m_max, seed)
    if total_mass is not None:
        m = rescale(m, total_mass)
    return np.ascontiguousarray(xy), np.ascontiguousarray(m)
