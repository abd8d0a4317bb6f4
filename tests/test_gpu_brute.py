"""Parity of the plain (brute-force) CUDA ray pass with the FP64 oracle.

Configuration C1 of the workload list: kappa_* = 0.3, kappa_s = 0, gamma = 0.3,
equal masses placed uniformly in the rectangular plane, a 128^2 map over
5 x 5 theta_E at 25 rays per unlensed pixel (1.04e7 rays).  Bars: deflection
<= 1e-5 theta_E, <= 1e-4 of rays binned differently.
"""
import numpy as np
import pytest

import oracle
from paper_2204_10871_gb300 import irs
from gpu_common import (C2, DEFLECTION_TOL, MISBIN_TOL, NEAR_LENS, c2_lenses, c2_oracle_rows, lenses_for,
                        misbinned, nearest_lens_distance, params_pair, ray_positions, require_gpu,
                        to_dev)

pytestmark = pytest.mark.gpu

C1 = dict(kappa_star=0.3, kappa_s=0.0, gamma=0.3, src=(-2.5, 2.5, -2.5, 2.5), npix=128, nav=25.0)


def _map_pair(torch, po, pl, xy, m):
    qo = oracle.size(po)
    co, mo, landed = oracle.make_map(po, qo, xy, m)
    with irs.Plan(pl) as plan:
        dxy, dm = to_dev(torch, xy, m)
        counts, mag = plan.make_map(dxy, dm)
        plan.sync()
        cg = counts.cpu().numpy()
        mg = mag.cpu().numpy()
    return qo, co, mo, landed, cg, mg


def test_sizing_matches_oracle():
    require_gpu()
    po, pl = params_pair(**C1)
    qo = oracle.size(po)
    with irs.Plan(pl) as plan:
        info = plan.info
    assert (info.n_rays_x, info.n_rays_y) == (qo.nrx, qo.nry)
    for a, b in [(info.lens_x0, qo.a1), (info.lens_x1, qo.a2), (info.lens_y0, qo.b1),
                 (info.lens_y1, qo.b2), (info.dx_ray, qo.dx3), (info.border, qo.border)]:
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b))


@pytest.mark.parametrize("n,rescale", [(61, False), (150, True)])
def test_c1_map_parity(n, rescale):
    torch = require_gpu()
    po, pl = params_pair(**C1)
    qo = oracle.size(po)
    xy, m = lenses_for(qo, n, seed=1, kappa_star=0.3 if rescale else None)
    qo, co, mo, landed, cg, mg = _map_pair(torch, po, pl, xy, m)
    assert cg.sum() <= qo.n_rays
    bad = misbinned(co, cg)
    assert bad <= MISBIN_TOL * landed, f"{bad} of {landed} rays binned differently"
    ratio = qo.dx3 ** 2 / (qo.sx * qo.sy)
    assert np.allclose(mg, cg.astype(np.float64) * ratio, rtol=1e-6)


def test_c1_sampled_deflection():
    torch = require_gpu()
    po, pl = params_pair(**C1)
    qo = oracle.size(po)
    xy, m = lenses_for(qo, 150, seed=1, kappa_star=0.3)
    rng = np.random.default_rng(2)
    idx = rng.integers(0, qo.n_rays, 4000).astype(np.int64)
    _, bo, po_pix = oracle.shoot_rays(po, qo, xy, m, idx)
    with irs.Plan(pl) as plan:
        dxy, dm = to_dev(torch, xy, m)
        beta, pix = plan.shoot_rays(dxy, dm, torch.from_numpy(idx).cuda())
        plan.sync()
    bg, pg = beta.cpu().numpy(), pix.cpu().numpy()
    err = np.abs(bg - bo).max(1)
    far = nearest_lens_distance(xy, ray_positions(qo, idx)) > NEAR_LENS
    assert far.sum() > 3000
    assert err[far].max() <= DEFLECTION_TOL, f"max deflection error {err[far].max():.3e}"
    # near lenses FP32 keeps ~1e-7 relative precision of the lens term
    assert np.all(err <= DEFLECTION_TOL * np.maximum(1.0, np.abs(bo).max(1)))
    assert np.mean(pg != po_pix) <= 2e-3


BRUTE_VARIANTS = range(16)


@pytest.mark.parametrize("variant", BRUTE_VARIANTS)
def test_every_brute_variant_meets_the_bars(variant):
    """Each kernel variant (rows per thread, rows sharing a reciprocal by
    pairs or by fours, packed rows, occupancy) against the FP64 oracle: the map (misbinned rays) and the
    sampled deflections, with 403 lenses so that several shared-memory stages
    and their TwoSum folds are exercised and the last stage carries massless
    padding lenses (its count rounded up to a multiple of 8)."""
    torch = require_gpu()
    po, pl = params_pair(**C1, kernel_variant=variant)
    qo = oracle.size(po)
    xy, m = lenses_for(qo, 403, seed=5, kappa_star=0.3)
    qo, co, mo, landed, cg, mg = _map_pair(torch, po, pl, xy, m)
    bad = misbinned(co, cg)
    assert bad <= MISBIN_TOL * landed, f"{bad} of {landed} rays binned differently"
    rng = np.random.default_rng(3)
    idx = rng.integers(0, qo.n_rays, 2000).astype(np.int64)
    _, bo, _ = oracle.shoot_rays(po, qo, xy, m, idx)
    with irs.Plan(pl) as plan:
        dxy, dm = to_dev(torch, xy, m)
        beta, _ = plan.shoot_rays(dxy, dm, torch.from_numpy(idx).cuda())
        plan.sync()
    err = np.abs(beta.cpu().numpy() - bo).max(1)
    far = nearest_lens_distance(xy, ray_positions(qo, idx)) > NEAR_LENS
    assert err[far].max() <= DEFLECTION_TOL, f"max deflection error {err[far].max():.3e}"


@pytest.mark.parametrize("npix,nav,n", [((7, 5), 9.3, 1), ((33, 17), 3.0, 255), ((16, 16), 4.0, 257),
                                        ((1, 1), 2000.0, 3)])
def test_ragged_sizes(npix, nav, n):
    """Lattices that fill no tile evenly, lens counts around the 256-lens stage."""
    torch = require_gpu()
    po, pl = params_pair(0.25, 0.1, -0.15, (-1.3, 0.7, -0.4, 1.1), npix, nav)
    qo = oracle.size(po)
    xy, m = lenses_for(qo, n, shape="uniform", seed=5)
    qo, co, mo, landed, cg, mg = _map_pair(torch, po, pl, xy, m)
    assert misbinned(co, cg) <= max(2, MISBIN_TOL * landed)


def test_lens_free_and_massless():
    """N_* = 0 and all-zero masses both give the lens-free sheet."""
    torch = require_gpu()
    po, pl = params_pair(0.3, 0.2, 0.1, (-1.0, 1.5, -1.2, 0.8), (24, 16), 37.0)
    qo = oracle.size(po)
    co, _, landed = oracle.make_map(po, qo, np.zeros((0, 2)), np.zeros(0))
    with irs.Plan(pl) as plan:
        counts, _ = plan.make_map(torch.zeros((0, 2), dtype=torch.float64, device="cuda"),
                                  torch.zeros(0, dtype=torch.float64, device="cuda"))
        xy = torch.rand((10, 2), dtype=torch.float64, device="cuda")
        counts0, _ = plan.make_map(xy, torch.zeros(10, dtype=torch.float64, device="cuda"))
        plan.sync()
    assert misbinned(co, counts.cpu().numpy()) <= max(2, MISBIN_TOL * landed)
    assert np.array_equal(counts.cpu().numpy(), counts0.cpu().numpy())


def test_circle_plane_point_lens():
    """Eq. (alpha), one unit lens at the centre of a circular plane (Paczynski)."""
    torch = require_gpu()
    po, pl = params_pair(0.0, 0.0, 0.0, (-2.0, 2.0, -2.0, 2.0), 40, 400.0, border=1.5,
                         plane=irs.IRS_PLANE_CIRCLE)
    qo, co, mo, landed, cg, mg = _map_pair(torch, po, pl, np.zeros((1, 2)), np.ones(1))
    assert misbinned(co, cg) <= MISBIN_TOL * landed


@pytest.mark.parametrize("src", [(1.0, 3.0, -2.5, -0.5), (-9.0, -5.0, 2.0, 6.5)])
def test_circle_plane_off_centre(src):
    """Eq. (alpha) for a circular plane centred away from the origin (the
    k_* theta_c term of the circle sheet is non-zero): map and sampled
    deflections against the oracle."""
    torch = require_gpu()
    po, pl = params_pair(0.3, 0.05, 0.25, src, 96, 16.3, plane=irs.IRS_PLANE_CIRCLE)
    qo = oracle.size(po)
    assert np.hypot(qo.cx, qo.cy) > 2.0
    xy, m = lenses_for(qo, 200, shape="uniform", seed=17, kappa_star=0.3, plane=irs.IRS_PLANE_CIRCLE)
    qo, co, mo, landed, cg, mg = _map_pair(torch, po, pl, xy, m)
    bad = misbinned(co, cg)
    assert bad <= MISBIN_TOL * landed, f"{bad} of {landed} rays binned differently"
    idx = np.random.default_rng(6).integers(0, qo.n_rays, 3000).astype(np.int64)
    _, bo, _ = oracle.shoot_rays(po, qo, xy, m, idx)
    with irs.Plan(pl) as plan:
        dxy, dm = to_dev(torch, xy, m)
        beta, _ = plan.shoot_rays(dxy, dm, torch.from_numpy(idx).cuda())
        plan.sync()
    err = np.abs(beta.cpu().numpy() - bo).max(1)
    far = nearest_lens_distance(xy, ray_positions(qo, idx)) > NEAR_LENS
    assert err[far].max() <= DEFLECTION_TOL, f"max deflection error {err[far].max():.3e}"


def test_c2_full_width_rows_vs_oracle():
    """The full mid-size workload (1e5 lenses, 2000^2 map, 100 rays/px): three
    whole lattice rows across the middle of the plane (1.0e6 rays, every ray
    summed over every lens by the oracle in FP64) against the same rows of the
    GPU brute force, at the misbinning bar."""
    torch = require_gpu()
    rows, co, landed = c2_oracle_rows()
    po, pl = params_pair(*C2, method=irs.IRS_BRUTE)
    qo = oracle.size(po)
    xy, m = c2_lenses(qo)
    with irs.Plan(pl) as plan:
        dxy, dm = to_dev(torch, xy, m)
        c = torch.zeros((2000, 2000), dtype=torch.uint32, device="cuda")
        irs.irs_make_map_rows(plan.handle, dxy, dm, rows[0], rows[1], c)
        plan.sync()
    cg = c.cpu().numpy()
    bad = misbinned(co, cg)
    print(f"\nbrute, rows {rows}: {bad} of {landed} rays binned differently ({bad / landed:.2e})")
    assert landed > 500000
    assert bad <= MISBIN_TOL * landed, f"{bad} of {landed} rays binned differently"


def test_repeat_is_deterministic():
    torch = require_gpu()
    po, pl = params_pair(**C1)
    qo = oracle.size(po)
    xy, m = lenses_for(qo, 150, seed=3, kappa_star=0.3)
    with irs.Plan(pl) as plan:
        dxy, dm = to_dev(torch, xy, m)
        a, _ = plan.make_map(dxy, dm)
        b, _ = plan.make_map(dxy, dm)
        plan.sync()
    assert torch.equal(a, b)


def test_bad_arguments_raise():
    torch = require_gpu()
    po, pl = params_pair(**C1)
    with irs.Plan(pl) as plan:
        xy = torch.zeros((5, 2), dtype=torch.float64, device="cuda")
        m = torch.ones(5, dtype=torch.float64, device="cuda")
        counts = torch.zeros((128, 128), dtype=torch.uint32, device="cuda")
        buf = torch.zeros(11, dtype=torch.float64, device="cuda")
        with pytest.raises(irs.IrsError):  # lens_xy not 16-byte aligned
            irs.irs_make_map(plan.handle, buf[1:], m, counts)
        with pytest.raises(ValueError):
            irs.irs_make_map(plan.handle, xy.float(), m, counts)
    for method, bad in ((irs.IRS_BRUTE, 16), (irs.IRS_BRUTE, -1), (irs.IRS_INTERP, 17)):
        _, p = params_pair(**C1, method=method, kernel_variant=bad)
        with pytest.raises(irs.IrsError):  # no such kernel variant
            irs.Plan(p)
