"""Helpers shared by the GPU parity tests: build/load the CUDA library, the
seeded workloads, and comparisons against the FP64 oracle."""
import functools

import numpy as np
import pytest

import oracle
from paper_2204_10871_gb300 import build as libbuild
from paper_2204_10871_gb300 import irs, lensgen

# Deflection bound of the plain ray pass (FP32 pairs) against the FP64 oracle,
# in Einstein radii, for rays whose nearest lens is farther than NEAR_LENS.
DEFLECTION_TOL = 1e-5
NEAR_LENS = 0.1
# Fraction of rays a brute-force map may bin into a different pixel.
MISBIN_TOL = 1e-4


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    libbuild.build()
    return torch


def params_pair(kappa_star, kappa_s, gamma, src, npix, nav, border=-1.0, plane=0,
                method=irs.IRS_BRUTE, **kw):
    """Matching oracle and library parameter structs; kw sets library-only
    fields (n_star, kernel_variant, cell_mult, ...)."""
    po = oracle.make_params(kappa_star, kappa_s, gamma, src, npix, nav, border=border, plane=plane)
    pl = irs.make_params(kappa_star, kappa_s, gamma, src, npix, nav, border=border, plane=plane,
                         method=method, **kw)
    return po, pl


def lenses_for(plan_o, n, shape="equal", seed=1, kappa_star=None, plane=0, m_min=0.1, m_max=1.0):
    """Seeded lens field in the oracle's plane; with kappa_star given, masses are
    rescaled so that the field's density is exactly kappa_star."""
    if plane == oracle.PLANE_CIRCLE:
        disc = (plan_o.cx, plan_o.cy, plan_o.circle_r)
        area = np.pi * plan_o.circle_r ** 2
        box = None
    else:
        disc = None
        area = plan_o.ix * plan_o.iy
        box = (plan_o.a1, plan_o.a2, plan_o.b1, plan_o.b2)
    total = kappa_star * area / np.pi if kappa_star is not None else None
    return lensgen.lens_field(n, box, shape=shape, seed=seed, total_mass=total, disc=disc,
                              m_min=m_min, m_max=m_max)


def to_dev(torch, xy, m):
    return (torch.from_numpy(np.ascontiguousarray(xy)).cuda(),
            torch.from_numpy(np.ascontiguousarray(m)).cuda())


def misbinned(counts_a, counts_b):
    """Lower bound of rays binned differently: half the L1 distance of the maps
    plus the rays one map kept and the other dropped."""
    a = counts_a.astype(np.int64)
    b = counts_b.astype(np.int64)
    d = np.abs(a - b).sum()
    kept = abs(int(a.sum()) - int(b.sum()))
    return (d - kept) / 2 + kept


def nearest_lens_distance(xy, t):
    if xy.shape[0] == 0:
        return np.full(t.shape[0], np.inf)
    d = np.full(t.shape[0], np.inf)
    for k in range(0, xy.shape[0], 4096):
        blk = xy[k:k + 4096]
        dd = np.hypot(t[:, None, 0] - blk[None, :, 0], t[:, None, 1] - blk[None, :, 1]).min(1)
        d = np.minimum(d, dd)
    return d


def ray_positions(plan_o, idx):
    i = idx % plan_o.nrx
    j = idx // plan_o.nrx
    return np.stack([plan_o.a1 + (i + 0.5) * plan_o.dx3, plan_o.b1 + (j + 0.5) * plan_o.dx3], 1)


# The mid-size workload (kappa_* = gamma = 0.45, 1e5 Salpeter lenses, 2000^2
# map over 20 x 20 theta_E, 100 rays per unlensed pixel) and a band of whole
# lattice rows across its middle that the oracle shoots in ~20 s on 16 cores
# (3 rows of 334,166 rays, every lens).
C2 = (0.45, 0.0, 0.45, (-10.0, 10.0, -10.0, 10.0), 2000, 100.0)
C2_N = 100000
C2_ROWS = 3


def c2_lenses(plan_o):
    return lenses_for(plan_o, C2_N, shape="salpeter", seed=2, kappa_star=C2[0])


@functools.lru_cache(maxsize=1)
def c2_oracle_rows():
    """(rows, oracle counts, landed) of the full-width band, computed once per
    test session."""
    po = oracle.make_params(*C2)
    qo = oracle.size(po)
    xy, m = c2_lenses(qo)
    r0 = qo.nry // 2
    rows = (r0, r0 + C2_ROWS)
    co, _, landed = oracle.make_map(po, qo, xy, m, rows=rows)
    return rows, co, landed
